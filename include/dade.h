/*
 * dade.h -- C ABI of libdade: DADE distance comparisons inside an IVF scan on
 * one GB300 (sm_103a).
 *
 * The method is DADE (Deng et al., "Efficient Data-aware Distance Comparison
 * Operations for High-Dimensional Approximate Nearest Neighbor Search"):
 * data objects are rotated once by the PCA basis W (Section 3.2, Eq. 10-12);
 * a distance comparison operation (DCO, Definition 1) between a query q and a
 * candidate o accumulates the squared distance over the leading dimensions in
 * steps of delta_d, forms the estimate dis'^2 = Lambda_D / Lambda_d * P_d
 * (Eq. 13) and rejects the candidate as soon as dis' > (1 + eps_d) r, where r
 * is the query's current K-th nearest distance and eps_d is set by the
 * significance level P_s (= alpha here) from sampled pairs (Section 3.3,
 * Eq. 14); a candidate that is never rejected gets its exact distance at
 * d = D (Algorithm 1).  IVF (Section 3.4) supplies the candidates: the
 * members of the nprobe inverted lists nearest to the query.
 *
 * Conventions for every entry point
 *   - Plain pointers and sizes only.  Row-major arrays.  Sizes are element
 *     counts unless named *_bytes.
 *   - Array arguments marked "host or device" may point to host memory
 *     (pageable or pinned) or to CUDA device memory; the library detects which
 *     and stages host data through its own device workspace.  Host results are
 *     complete when the call returns; device results are complete when work
 *     queued on `stream` before the next synchronisation has finished.
 *   - The caller owns every array it passes; the library owns the index.
 *   - Nothing throws across the ABI.  Every failure returns a dade_status and
 *     leaves a message for dade_last_error() (thread-local).  Invalid
 *     arguments are rejected before any GPU work is queued.
 *   - All GPU work runs on `stream` (a cudaStream_t; NULL = legacy default).
 *     One index serves one call at a time: concurrent calls on the same index
 *     from several host threads are not supported (they share its workspace).
 *   - Distances returned are squared Euclidean distances (monotone in the
 *     paper's dis; no square root on the hot path).  Result lists are ordered
 *     by (squared distance, id) ascending; slots beyond the candidates found
 *     hold id -1 and distance +inf.
 */
#ifndef DADE_H
#define DADE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dade_index dade_index;      /* opaque; resident in device memory */
typedef struct CUstream_st *dade_stream;   /* same type as cudaStream_t */

typedef enum {
    DADE_OK = 0,
    DADE_EINVAL = 1,        /* an argument is out of range or inconsistent */
    DADE_ENOMEM = 2,        /* a host or device allocation failed */
    DADE_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    DADE_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
    DADE_EUNSUPPORTED = 5,  /* valid request the library does not implement */
    DADE_EIO = 6,           /* file could not be read or written */
    DADE_ECANCELLED = 7     /* a server request was cancelled (dade_server_cancel) */
} dade_status;

enum {
    DADE_MAX_DIM = 1024,    /* D <= 1024 */
    DADE_MAX_K = 256,       /* K <= 256 */
    DADE_BLOCK = 16         /* dimensions per stored block; delta_d is a multiple */
};

/* Threshold schedule / DCO kind of a search. */
typedef enum {
    DADE_MODE_DADE = 0,     /* Algorithm 1 with the Section 3.3 test */
    DADE_MODE_FD = 1        /* FDScanning (Section 4.1): exact full-D distance for every candidate */
} dade_mode;

/*
 * Threshold schedule of a DADE search.  Lists are scanned in probe order and
 * each list in tiles of opts->tile candidates (ascending base id; a tile
 * never spans two lists).  Every candidate of a tile is tested against the
 * K-th distance r held when the tile starts:
 *   DADE_SCHED_TILE       r after all earlier tiles (tile-synchronous; default);
 *   DADE_SCHED_PIPELINED  r after all tiles but the n_inc - 1 just before it,
 *                         where n_inc = ceil(ceil(D/16) / (delta_d/16)) is the
 *                         number of increments: up to n_inc tiles are in flight
 *                         at once, one per increment.  Used when n_inc <= 8,
 *                         otherwise the tile schedule runs.
 *   DADE_SCHED_SEEDED     the first opts->seed_lists probed lists as in
 *                         DADE_SCHED_TILE; every candidate of the later lists
 *                         is tested against r frozen after those lists.  The
 *                         later lists are then scanned list-major where the
 *                         list-major kernels apply (D > 112 and delta_d of 16,
 *                         32, 64 or 128 dims): each list's rows are staged
 *                         once for all the queries probing it (one persistent
 *                         launch over (list chunk, query group) items), and
 *                         the K nearest are merged at the end.  Any other D or
 *                         delta_d, and DADE_FLAG_SEED_SPLIT, scan them
 *                         query-major, each query's later lists split over
 *                         several thread blocks.  Every D and delta_d is
 *                         served, with the same results either way.
 *   DADE_SCHED_ROUNDS     rows instead of lists: round e holds rows
 *                         [R_e, R_{e+1}) of every probed list, with R_0 = 0,
 *                         R_1 = opts->tile (any tile >= 1) and R_{e+1} = 2 R_e,
 *                         and every candidate of round e is tested against r
 *                         after rounds 0..e-1 (round 0: r = +inf, so its
 *                         candidates get exact distances).  Every list
 *                         advances through the same row windows, so a long
 *                         list is scanned in doubling windows, each split into
 *                         chunks over many thread blocks, while r tightens
 *                         between the windows.  Each round runs list-major
 *                         where the list-major kernels apply (see
 *                         DADE_SCHED_SEEDED), else, and with
 *                         DADE_FLAG_SEED_SPLIT or DADE_FLAG_LEAD, query-major
 *                         split over thread blocks; same results either way.
 *                         For indexes whose list sizes are very uneven.
 * A staler threshold can only prune less.  FDScanning results do not depend
 * on the schedule.
 */
typedef enum {
    DADE_SCHED_TILE = 0,
    DADE_SCHED_PIPELINED = 1,
    DADE_SCHED_SEEDED = 2,
    DADE_SCHED_ROUNDS = 3
} dade_schedule;

/* dade_search_opts.flags */
enum {
    DADE_FLAG_GENERIC_KERNEL = 1,  /* skip the kernels specialised for D <= 128 (testing) */
    DADE_FLAG_LEAD = 2,            /* prefilter the first increment on the index's low-precision copy
                                      (DADE mode, tile schedule, min(delta_d, D_pad) <= lead_dims) */
    DADE_FLAG_QUERY_ORDER = 4,     /* run the queries grouped by their first probed list (results are
                                      the same in any order; grouped, they share list rows in L2) */
    DADE_FLAG_ROW_TAIL = 8,        /* a candidate that survives the first increment reads its dims from
                                      tail_from on from the index's row-major copy: one contiguous row
                                      instead of one 64-byte piece per 16-dim slab.  Same results. */
    DADE_FLAG_TC_PREFILTER = 32,   /* list-major passes (DADE_SCHED_SEEDED, DADE_SCHED_ROUNDS; D > 112,
                                      delta_d of 16, 32 or 64 dims): the first increment's inner products
                                      q'.o' on the tensor cores (the FP32 rows read as TF32, the query
                                      split into two TF32 parts), and a certified lower bound of each
                                      partial distance; a candidate is dropped only where the bound
                                      exceeds the threshold by more than the FP32 path's rounding, every
                                      other one runs the FP32 path.  Same results; opts->lead_stats
                                      counts the candidates the bound dropped. */
    DADE_FLAG_SEED_SPLIT = 16,     /* DADE_SCHED_SEEDED: every pass with r frozen (the lists after the
                                      seeds; with whole-list tiles, each seed epoch too) runs query-major
                                      on the tile kernel, each query's lists split into parts over
                                      several thread blocks (the candidates are independent there),
                                      instead of list-major.  Same tests and thresholds.  The same for
                                      every round of DADE_SCHED_ROUNDS. */
    DADE_FLAG_CHECK_TIMEOUT = 64   /* check of the failure path: the first wait on a copy of every thread
                                      block of the scan waits instead on a device word that nothing
                                      sets, so it runs out after wait_ns with the block's first copies in
                                      flight.  The blocks let those copies land and leave; dade_sync
                                      returns DADE_ETIMEOUT and the index serves the next search.  The
                                      results of that search are undefined. */
};

/*
 * Low-precision copy of the leading dimensions, a conservative prefilter for
 * the first increment of a search (DADE_FLAG_LEAD).  The paper reads FP32
 * throughout; this copy is an addition of this library.  For base vector o
 * in list c the index stores, over the first lead_dims rotated dims, the
 * residual r = o' - c' quantised (BF16 round to nearest even, or FP8 e4m3
 * of r / s with one FP32 scale s per (list, 16-dim block), saturating), and
 * per 16-dim block b the error norm e_b = || r - dequant(code) || over the
 * blocks 0..b (FP64, rounded up).  By the triangle inequality the exact
 * partial distance satisfies sqrt(P_d) >= sqrt(P~_d) - e, with P~_d formed
 * from q' - c' and the dequantised codes.  The scan drops a candidate at the
 * first increment only when that lower bound, less FP32 rounding, exceeds
 * coef_d r^2 (Section 3.3 test) with a margin above rounding, so the exact
 * test would drop it too; every other candidate reloads its FP32 rows and
 * runs Algorithm 1 from the first increment.  Results and per-query
 * statistics equal those of the FP32 path; only the bytes read change.
 * Extra memory: lead_dims * (2 B BF16 | 1 B FP8) + 4 * lead_dims / 16 B per
 * vector (padded slots included).
 */
typedef enum {
    DADE_LEAD_NONE = 0,
    DADE_LEAD_BF16 = 1,        /* bfloat16, round to nearest even */
    DADE_LEAD_FP8 = 2          /* FP8 e4m3 with one FP32 scale per (list, 16-dim block) */
} dade_lead_format;

/*
 * The orthogonal transformation of an index.  DADE's is the PCA basis with
 * descending eigenvalues (Section 3.2).  The comparator ADSampling (Gao et
 * al., the paper's baseline) uses a random orthogonal transformation instead:
 * DADE_TRANSFORM_RANDOM draws a Haar-distributed one from `seed`
 * (Gram-Schmidt of SplitMix64 Gaussians), DADE_TRANSFORM_GIVEN takes `basis`.
 * lambda_k is then the data's variance along w_k (in the given order).
 */
typedef enum {
    DADE_TRANSFORM_PCA = 0,
    DADE_TRANSFORM_RANDOM = 1,
    DADE_TRANSFORM_GIVEN = 2
} dade_transform;

/*
 * Distance estimator and test of a search.  DADE: dis'^2 = Lambda_D/Lambda_d
 * P_d (Eq. 13), prune iff dis' > (1 + eps_d) r with eps_d from the sampled
 * pairs at significance alpha (Eq. 14).  ADSampling: dis'^2 = (D/d) P_d,
 * prune iff dis' > (1 + eps0 / sqrt(d)) r, eps0 = opts->eps0 (data-oblivious;
 * meant for an index with a random transformation).  FDScanning: opts->mode.
 */
typedef enum {
    DADE_ESTIMATOR_DADE = 0,
    DADE_ESTIMATOR_ADSAMPLING = 1
} dade_estimator;

/* Index construction options.  Zero-initialise, then call dade_build_opts_default(). */
typedef struct {
    int32_t n_clusters;        /* N_c, number of inverted lists (>= 1) */
    int32_t kmeans_iters;      /* Lloyd iterations (default 10); ignored when assign != NULL */
    uint64_t seed;             /* key of the SplitMix64 draws used when kmeans_init / pairs are NULL */
    int64_t eps_pairs;         /* M, sampled pairs for eps_d (default 100000) */
    const int32_t *assign;     /* host, optional [n]: list of every base vector (0..n_clusters-1);
                                  list centroids become member means; no k-means runs */
    const int64_t *kmeans_init;/* host, optional [n_clusters]: distinct base ids that seed k-means */
    const int64_t *pairs;      /* host, optional [2 * eps_pairs]: pair ids (i != j) for eps_d */
    int32_t lead_format;       /* dade_lead_format: extra low-precision copy of the leading dims */
    int32_t lead_dims;         /* leading dims in that copy (multiple of 16, <= D; 0 = none) */
    int32_t tail_from;         /* keep a row-major FP32 copy of dims [tail_from, D) of every vector
                                  (multiple of 16, < D; 0 = none), see DADE_FLAG_ROW_TAIL */
    int32_t transform;         /* dade_transform (default DADE_TRANSFORM_PCA) */
    const double *basis;       /* host, optional [d * d] orthonormal columns (W[j*d + k] = component j of
                                  w_k) for DADE_TRANSFORM_GIVEN */
    int32_t reserved[2];
} dade_build_opts;

/* Search options; NULL means all defaults. */
typedef struct {
    int32_t mode;              /* dade_mode (default DADE_MODE_DADE) */
    int32_t tile;              /* candidates per threshold refresh (default 128; 32..256, multiple of 32;
                                  DADE_SCHED_SEEDED also takes any tile >= the longest list: every seed
                                  list is then one epoch and runs list-major too; DADE_SCHED_ROUNDS:
                                  rows of every list in the first round, any value >= 1) */
    int64_t *stats;            /* device, optional [nq * 4]: per query candidates scanned, sum of
                                  dimensions used, candidates accepted by the DCO, candidates pruned */
    int32_t spec;              /* tile schedule: 16-dim blocks of a candidate that survived the first
                                  increment loaded together ahead of its tests (1..8, default 8) */
    int32_t threads;           /* threads per query's CTA: 0 (default 128), 128 or 256 */
    int32_t schedule;          /* dade_schedule (default DADE_SCHED_TILE) */
    int32_t flags;             /* DADE_FLAG_* bits */
    int64_t *lead_stats;       /* device, optional [nq]: candidates dropped by the low-precision prefilter
                                  (DADE_FLAG_LEAD) or by the tensor-core prefilter (DADE_FLAG_TC_PREFILTER) */
    int32_t seed_lists;        /* DADE_SCHED_SEEDED: lists scanned before r is frozen (0: 2; >= nprobe:
                                  the tile schedule) */
    int32_t estimator;         /* dade_estimator (default DADE_ESTIMATOR_DADE) */
    float eps0;                /* ADSampling's eps0 (> 0) */
    int32_t stage_dims;        /* tile schedule, any D: dims of every candidate of a tile streamed into
                                  shared memory at once (0: delta_d; else a multiple of delta_d), tested
                                  at each increment inside; survivors then gather the rest.  Same
                                  results; a deeper stage trades gathers for streaming when most
                                  candidates outlive the first increments. */
    int32_t list_chunk;        /* list-major passes of DADE_SCHED_SEEDED and DADE_SCHED_ROUNDS: rows of one list per work
                                  item (0: 4096; else a multiple of 64); a long list becomes several
                                  items run by different thread blocks.  Same results. */
    int32_t stage_ring;        /* tile kernel for any D: staged tiles in flight per thread block (0: 2;
                                  2..8); deeper rings hide more load latency for more shared memory.
                                  Same results. */
    int64_t wait_ns;           /* limit, in ns, of every bounded device-side wait of the scan kernels for a
                                  copy or an MMA (0: 2 s).  A wait that runs out makes its thread block
                                  record DADE_ETIMEOUT (reported by dade_sync or by the call, for host
                                  outputs), let its copies in flight land (bounded), free what it holds
                                  and leave; that query's results are then undefined, the index stays
                                  usable.  Limits below 0.2 ms poll without suspending, limits below
                                  1 us poll once. */
    int32_t tc_min_rows;       /* DADE_FLAG_TC_PREFILTER under DADE_SCHED_ROUNDS: a round whose row window
                                  is shorter runs the FP32 list-major kernel instead (its work items are
                                  a few tiles, where the copy-MMA-read chain costs more than the bound
                                  saves); 0: every round after the first.  Results are the same. */
} dade_search_opts;

/* Description of a built index. */
typedef struct {
    int64_t n;                 /* base vectors */
    int32_t d;                 /* dimension D */
    int32_t d_pad;             /* D rounded up to a multiple of 16 (storage width) */
    int32_t n_clusters;
    int32_t max_list;          /* longest inverted list */
    int64_t eps_kept;          /* sampled pairs kept for eps_d (nonzero distance) */
    int64_t device_bytes;      /* device memory held by the index (excluding workspace) */
    int64_t data_bytes;        /* packed rotated vectors */
    int32_t kmeans_iters;      /* Lloyd iterations run (0 when lists were given) */
    int32_t lead_format;       /* dade_lead_format of the index */
    int32_t lead_dims;
    int32_t tail_from;         /* 0 or the first dim of the row-major copy */
} dade_info;

/* Fields for dade_index_export (host copies, for inspection and tests). */
typedef enum {
    DADE_FIELD_MEAN = 0,       /* double [d]          mu */
    DADE_FIELD_BASIS = 1,      /* double [d * d]      W, column k = w_k (row-major: W[j*d + k]) */
    DADE_FIELD_EIGVAL = 2,     /* double [d]          lambda_1 >= ... >= lambda_D */
    DADE_FIELD_CENTROIDS = 3,  /* float  [n_clusters * d]  rotated list centroids */
    DADE_FIELD_ASSIGN = 4,     /* int32  [n]          list of every base vector */
    DADE_FIELD_ROTATED = 5,    /* float  [n * d]      rotated base vectors, by base id */
    DADE_FIELD_RHO = 6,        /* double [(d_pad/16 - 1) * eps_kept]  sorted rho_d samples, row t is d = 16 (t+1) */
    DADE_FIELD_KMEANS_OBJ = 7, /* double [kmeans_iters] objective of each assignment step */
    DADE_FIELD_LEAD_DEQ = 8,   /* float  [n * lead_dims] dequantised lead residuals, by base id */
    DADE_FIELD_LEAD_ERR = 9,   /* float  [lead_dims/16 * n] row b: error norm over blocks 0..b, by base id */
    DADE_FIELD_LEAD_SCALE = 10 /* float  [n_clusters * lead_dims/16] FP8 block scales (1 for BF16) */
} dade_field;

void dade_build_opts_default(dade_build_opts *opts);

/*
 * Build an index over n base vectors of dimension d (Section 3.2 and 3.4):
 *   mean and covariance of the data (FP64 on the GPU), eigendecomposition
 *   (FP64 on the host), rotation o' = W^T (o - mu) of every vector (FP32 on
 *   the GPU), inverted lists (given `assign`, or seeded k-means on the rotated
 *   vectors), and the sorted rho_d sample for eps_d (Eq. 14) at every d that is
 *   a multiple of 16 below D.  Vectors are stored rotated, once, in a
 *   dimension-blocked layout: per list, per 16-dimension block, a contiguous
 *   [list length][16] FP32 slab.
 * base: host or device, [n * d] FP32.  n >= 2, 1 <= d <= DADE_MAX_DIM,
 * 1 <= n_clusters <= n.  On success *out receives the index (free it with
 * dade_free_index).  Synchronises `stream` before returning.
 */
dade_status dade_build_index(const float *base, int64_t n, int32_t d, const dade_build_opts *opts,
                             dade_index **out, dade_stream stream);

/* Release an index and its workspace.  NULL is ignored. */
void dade_free_index(dade_index *ix);

/*
 * A query step captured into a CUDA graph (no counterpart in the paper; a
 * launch-overhead device for small, repeated batches).  dade_graph_create
 * runs dade_query(ix, q, nq, k, nprobe, alpha, delta_d, opts, ids, dists)
 * once, then captures the same call on a private stream; q, ids, dists (and
 * opts->stats, opts->lead_stats if set) must be device buffers, and stay
 * bound to the graph: a launch reads whatever q holds at that time and
 * overwrites ids and dists.  The graph uses the index's workspace: launch it
 * while no other call on the same index is in flight, and free it before the
 * index.  dade_graph_launch enqueues one replay on `stream`.  Errors:
 * DADE_EINVAL (host buffers, bad arguments), DADE_ECUDA (capture refused).
 */
typedef struct dade_graph dade_graph;
dade_status dade_graph_create(const dade_index *ix, const float *q, int64_t nq, int32_t k, int32_t nprobe,
                              float alpha, int32_t delta_d, const dade_search_opts *opts, int64_t *ids, float *dists,
                              dade_graph **out);
dade_status dade_graph_launch(dade_graph *g, dade_stream stream);
void dade_graph_free(dade_graph *g);

/*
 * Continuous-batching request server over one resident index (no counterpart
 * in the paper).  Requests (host queries with their own K, nprobe, alpha,
 * delta_d) are queued by dade_server_submit and admitted by a dispatcher
 * thread into slots as slots free up: each slot is a CUDA stream with its
 * own device workspace and pinned buffers, so batches in different slots
 * overlap on the GPU.  A batch is the oldest pending request plus every
 * later pending request it can run with, up to max_batch queries: under the
 * tile schedule, and the row rounds where they run list-major, every request
 * with the same alpha and delta_d (mixed K and nprobe run in one launch,
 * dade_query_mixed), otherwise the same K, nprobe, alpha and delta_d.  Every query's result depends only on
 * that query, so a request gets the same result alone and in any mix.  With
 * a device_budget, admission is by bytes: a batch starts only while every
 * slot's staging buffers plus the workspace the slots' batches grew to (an
 * estimate from the batch's queries, largest K and largest nprobe) stay
 * within the budget; a request that cannot fit even alone completes with
 * DADE_ENOMEM.  The caller's query and result buffers must stay valid until
 * dade_server_wait returns for the ticket (or dade_server_cancel returns).
 * dade_server_free drains the queue and the slots.
 */
typedef struct dade_server dade_server;
typedef struct {
    int32_t slots;             /* batches in flight on the GPU at once (default 4) */
    int32_t max_batch;         /* queries per batch, and per request (default 1024) */
    int32_t max_k;             /* largest K of a request (default 100) */
    int32_t max_nprobe;        /* largest nprobe of a request (default 128) */
    int64_t device_budget;     /* device bytes of the server: slots' staging buffers and the workspace
                                  admitted batches grow (0: no limit); fewer slots if even one request
                                  would not fit beside their staging buffers */
    int32_t mode, tile, threads, schedule, seed_lists, flags;   /* dade_search_opts of every batch */
    int32_t stage_dims;        /* dade_search_opts.stage_dims of every batch (0: delta_d) */
    int32_t list_chunk;        /* dade_search_opts.list_chunk of every batch (0: 4096) */
    int32_t tc_min_rows;       /* dade_search_opts.tc_min_rows of every batch (0: every round after the first) */
    int32_t reserved;
} dade_server_opts;
typedef struct {
    int64_t slots, slot_bytes;          /* slots created, device bytes of a slot running a full batch */
    int64_t requests, requests_done;    /* submitted, completed */
    int64_t batches, queries;           /* batches launched, queries in them */
    int64_t max_inflight;               /* most batches on the GPU at once */
} dade_server_stats;
void dade_server_opts_default(dade_server_opts *o);
dade_status dade_server_create(const dade_index *ix, const dade_server_opts *opts, dade_server **out);
/* Queue a request: q host [nq * d] raw queries; ids, dists host [nq * k], written before the ticket completes. */
dade_status dade_server_submit(dade_server *s, const float *q, int64_t nq, int32_t k, int32_t nprobe, float alpha,
                               int32_t delta_d, int64_t *ids, float *dists, uint64_t *ticket);
/* Wait for a ticket (timeout_ms < 0: no limit; DADE_ETIMEOUT if it expires, the ticket stays valid).
 * latency_s (may be NULL): seconds from submit to completion. */
dade_status dade_server_wait(dade_server *s, uint64_t ticket, int64_t timeout_ms, double *latency_s);
/* Cancel a request: a pending one leaves the queue, one in flight runs on but its results are not
 * written to the caller's buffers; either way dade_server_wait returns DADE_ECANCELLED for it (and the
 * caller's buffers are free once cancel returns).  DADE_EINVAL for an unknown or completed ticket. */
dade_status dade_server_cancel(dade_server *s, uint64_t ticket);
/* A native load generator for measuring the server (no counterpart in the paper): request i is one
 * query, q host [n * d] row i, with k[i] and nprobe[i], submitted from the calling thread at
 * arrival_s[i] seconds after the call starts (non-decreasing; the thread spins until then), then
 * every ticket is waited for.  ids, dists: host [n * k_stride], row i holding request i's k[i]
 * results; latency_s: host [n], submit to completion (-1 if refused); submit_s (may be NULL): the
 * seconds the submission took.  Returns the first error of any request (the others still run). */
dade_status dade_server_replay(dade_server *s, const float *q, int64_t n, const int32_t *k, const int32_t *nprobe,
                               float alpha, int32_t delta_d, const double *arrival_s, int32_t k_stride, int64_t *ids,
                               float *dists, double *latency_s, double *submit_s);
dade_status dade_server_stats_get(dade_server *s, dade_server_stats *out);
void dade_server_free(dade_server *s);

/*
 * Write a built index to `path` as one binary file (this library's own
 * format, version 1, little-endian; the paper stores no index): the FP64
 * offline results (mean, basis, eigenvalues, rho_d sample), the list
 * assignment and descriptors, and the device arrays (centroids, packed
 * vectors, ids, the optional low-precision leading blocks).
 * Synchronous; the index is unchanged.  DADE_EIO if the file cannot be
 * written.
 */
dade_status dade_save_index(const dade_index *ix, const char *path);

/*
 * Read an index written by dade_save_index onto the current device.  Every
 * size is checked against the header and every list descriptor and slot id
 * against the arrays it indexes before use: a damaged or foreign file gives
 * DADE_EINVAL (DADE_EIO if unreadable or truncated) and no index.
 * Synchronous.  The caller frees the result with dade_free_index.
 */
dade_status dade_load_index(const char *path, dade_index **out);

/*
 * ---- The index split by inverted lists (one shard per GPU) -------------------
 * The IVF search of Section 3.4 visits whole inverted lists, so the lists can
 * be dealt to G shards: each shard keeps the mean, the basis, the eigenvalue
 * sums and the rho_d sample (so eps_d and the coefficients of the Section 3.3
 * test are the full index's, Eq. 13-14) and every centroid (so every shard
 * probes the same global lists), but only the rows of its own lists.  A
 * search on a shard is the IVF loop over the probed lists it holds, with its
 * own threshold r (the K-th distance among those lists: never below the
 * unsharded search's r, so it prunes no more than that search would, and a
 * stale r is safe).  The sharded result is the K nearest of the G shards'
 * results, merged by dade_merge_shards.  In FD mode it equals the unsharded
 * result exactly; in DADE mode it equals the merge of the per-shard searches.
 */

/*
 * Deal n_lists lists of list_rows[c] rows to n_shards shards, balanced by
 * rows: longest list first (ties by list id), each to the shard with the
 * fewest rows so far (ties by the lower shard id).  Host only (no device
 * call); deterministic, so every rank computes the same owner[] from the
 * same sizes.  list_rows: host [n_lists] (>= 0); owner: host [n_lists],
 * written with 0 .. n_shards - 1.  DADE_EINVAL on a NULL pointer, n_lists
 * or n_shards < 1, or a negative size.
 */
dade_status dade_shard_lists(const int64_t *list_rows, int32_t n_lists, int32_t n_shards, int32_t *owner);

/*
 * A new index on the current device holding shard `shard` of ix: the lists
 * c with owner[c] == shard keep their rows, ids and optional copies
 * (low-precision lead, row-major tail); every other list is empty.
 * Everything else is copied from ix (see above), so the shard's rotation,
 * probe and eps table equal ix's.  owner: host [n_clusters] (from
 * dade_shard_lists or the caller's own partition).  The shard keeps ix's id
 * space: dade_index_info reports ix's n, and dade_index_export of the
 * per-vector fields gives zeros for the vectors it does not hold.  A shard
 * cannot be saved (dade_save_index returns DADE_EINVAL) or split again.
 * Synchronous; ix is unchanged.  The caller frees the result with
 * dade_free_index.
 */
dade_status dade_index_subset(const dade_index *ix, const int32_t *owner, int32_t shard, dade_index **out);

/*
 * Merge the results of n_shards searches of the same nq queries into the K
 * nearest.  ids, dists: device [n_shards][nq][k] (shard-major, as an
 * all-gather of the shards' [nq][k] results lays them out), each shard's row
 * ascending by (distance, id) as dade_search writes it, empty places id -1 at
 * +inf; out_ids, out_dists: device [nq][k], the k smallest (distance, id)
 * pairs of the shards' rows, ascending (ties by id, then by shard).  A list
 * that is on one shard only gives every id at most once.  Asynchronous on
 * `stream`.  DADE_EINVAL on host buffers, NULL pointers or sizes out of range
 * (1 <= k <= DADE_MAX_K, n_shards >= 1).
 */
dade_status dade_merge_shards(const int64_t *ids, const float *dists, int32_t n_shards, int64_t nq, int32_t k,
                              int64_t *out_ids, float *out_dists, dade_stream stream);

/*
 * Query rotation q' = W^T (q - mu) (Lemma 1, Section 3.2): the transformed
 * query that Algorithm 1 takes as input.  q: host or device [nq * d] FP32;
 * q_rot: host or device [nq * d] FP32 output.  nq = 0 is a no-op.
 */
dade_status dade_rotate_queries(const dade_index *ix, const float *q, int64_t nq, float *q_rot,
                                dade_stream stream);

/*
 * IVF probe (Section 3.4): for every rotated query, the ids of the nprobe
 * lists whose centroids are nearest, ordered by (squared distance, list id).
 * q_rot: host or device [nq * d]; probe: host or device [nq * nprobe] int32.
 */
dade_status dade_probe(const dade_index *ix, const float *q_rot, int64_t nq, int32_t nprobe,
                       int32_t *probe, dade_stream stream);

/*
 * DADE-IVF search on rotated queries: probe, then scan the probed lists with
 * one DCO per candidate (Algorithm 1 and the Section 3.3 test at
 * significance alpha) against the query's current K-th distance, keeping the
 * K nearest.  Lists are scanned in probe order, members in ascending base id,
 * in tiles of opts->tile candidates, each tile tested against the K-th
 * distance of the threshold schedule opts->schedule (see dade_schedule).
 * q_rot: host or device [nq * d]; ids: host or device [nq * k] int64; dists:
 * host or device [nq * k] FP32 squared distances.  1 <= k <= DADE_MAX_K,
 * 1 <= nprobe <= n_clusters, 0 < alpha < 1, delta_d a multiple of 16 in
 * [16, DADE_MAX_DIM].  alpha and delta_d are ignored in DADE_MODE_FD.
 */
dade_status dade_search(const dade_index *ix, const float *q_rot, int64_t nq, int32_t k,
                        int32_t nprobe, float alpha, int32_t delta_d, const dade_search_opts *opts,
                        int64_t *ids, float *dists, dade_stream stream);

/*
 * The scan step alone: DADE (or FDScanning) over given probe lists, e.g. the
 * output of dade_probe or of another candidate generator.  probe: host or
 * device [nq * nprobe] int32 list ids, each in 0..n_clusters-1, scanned in
 * the order given.  Other arguments, limits and outputs as dade_search.
 */
dade_status dade_scan(const dade_index *ix, const float *q_rot, const int32_t *probe, int64_t nq, int32_t k,
                      int32_t nprobe, float alpha, int32_t delta_d, const dade_search_opts *opts, int64_t *ids,
                      float *dists, dade_stream stream);

/*
 * Tune a scan shape: time, on the caller's batch, the execution options that
 * leave the results unchanged -- opts->threads (128 or 256) and the flags
 * DADE_FLAG_QUERY_ORDER, DADE_FLAG_ROW_TAIL (index built with tail_from) and,
 * for DADE_SCHED_SEEDED, DADE_FLAG_SEED_SPLIT -- and write the fastest into
 * *opts (every other field is kept).  The choice is cached per index and
 * shape (nq, k, nprobe, alpha, delta_d and the result-changing options): a
 * repeated shape returns at once.  q_rot, probe, ids and dists must be device
 * buffers (ids and dists are scratch here and hold the last timed run's
 * results); synchronous on `stream`.  DADE_EINVAL for NULL or host buffers.
 */
dade_status dade_tune(const dade_index *ix, const float *q_rot, const int32_t *probe, int64_t nq, int32_t k,
                      int32_t nprobe, float alpha, int32_t delta_d, dade_search_opts *opts, int64_t *ids,
                      float *dists, dade_stream stream);

/*
 * ---- Operating point for a recall target (library autotuner) -------------------
 * The paper fixes P_s (alpha) and delta_d by hand (Section 4.1) and sweeps
 * nprobe for its recall-QPS curves.  dade_autotune finds, on the caller's
 * sample of queries and their exact K nearest ids, the fastest point whose
 * recall@K reaches a target: the smallest rung of an nprobe ladder at which
 * FDScanning (exact distances of the probed lists, the best any DCO can
 * return there) reaches the target, and the next two rungs; at each, delta_d
 * in {16, 32, 64} (<= D_pad), the execution variants the index serves (tile
 * schedule, with the low-precision prefilter when the index has the copy;
 * seeded schedule with 2 or 3 seed lists, later lists list-major or split over
 * thread blocks; row rounds from 16 or 32 rows with
 * work items of the default size or of 1,024 rows, and with the tensor-core
 * prefilter where D > 112), and alpha from 0.98
 * down to 0.05 until the recall is reached; every passing point is timed
 * (dade_probe + dade_scan, CUDA events on `stream`) and the fastest kept,
 * then dade_tune adds the result-neutral options.  The result is cached in
 * the process and, with cache_path, appended to a JSON-lines file (one flat
 * object per line), keyed by a fingerprint of the index (sizes, eigenvalues,
 * list sizes, copies), K, the recall target, the sample size (power-of-two
 * bucket) and the GPU (name, SM count); a later call with the same key
 * returns the cached point without timing anything (from_cache = 1).
 */
enum {
    DADE_AUTOTUNE_FORCE = 1    /* sweep even when the cache holds the key (and append the new point) */
};

typedef struct {
    float recall_target;       /* recall@K the point must reach on the queries given (default 0.95) */
    int32_t n_nprobe;          /* entries of nprobe_ladder; 0: 4, 6, 8, 10, 12, 16, ... up to min(N_c, 512) */
    const int32_t *nprobe_ladder;  /* host [n_nprobe], ascending, within 1 .. n_clusters */
    int32_t reps;              /* timed runs per point (default 3) */
    int32_t flags;             /* DADE_AUTOTUNE_* */
    const char *cache_path;    /* JSON-lines cache file, read and appended (NULL: the process cache only) */
    int32_t reserved[4];
} dade_autotune_opts;

typedef struct {
    int32_t nprobe, delta_d;
    float alpha;
    dade_search_opts opts;     /* mode, schedule, tile, seed_lists, list_chunk, threads, flags of the point;
                                  stats and lead_stats NULL */
    float recall;              /* recall@K on the queries given */
    float ms;                  /* mean time of probe + scan of the queries given */
    int32_t from_cache;        /* 1: returned from the cache, nothing was timed */
    int32_t points_tried;      /* searches run by the sweep */
} dade_autotune_result;

void dade_autotune_opts_default(dade_autotune_opts *opts);

/*
 * q: host or device [nq * d] raw queries (rotated by the call); gt_ids: host
 * [nq * k], each query's exact K nearest base ids (any order).  Synchronous
 * on `stream`; allocates its scratch on the device (the allocation hook
 * applies).  DADE_EINVAL on NULL pointers, a device gt_ids, sizes out of
 * range or a ladder that does not ascend within 1 .. n_clusters;
 * DADE_EUNSUPPORTED when no point of the ladder reaches the target (the
 * message says whether the exact scan does).
 */
dade_status dade_autotune(const dade_index *ix, const float *q, int64_t nq, int32_t k, const int64_t *gt_ids,
                          const dade_autotune_opts *opts, dade_autotune_result *out, dade_stream stream);

/*
 * End-to-end query: dade_rotate_queries followed by dade_search, on raw
 * queries.  q: host or device [nq * d].  Same outputs and limits as
 * dade_search.  With host buffers the call copies inputs in and results out
 * and returns when the results are on the host.
 */
dade_status dade_query(const dade_index *ix, const float *q, int64_t nq, int32_t k, int32_t nprobe,
                       float alpha, int32_t delta_d, const dade_search_opts *opts, int64_t *ids,
                       float *dists, dade_stream stream);

/*
 * dade_query with a K and an nprobe per query (the paper's IVF search,
 * Section 3.4, run for each query with its own K and nprobe): one rotation,
 * one probe of the nprobe_max nearest lists (a query's first nprobe[i] of
 * them, in (distance, id) order, are its own nprobe[i] nearest) and one scan
 * launch in which query i keeps its k[i] nearest, tests against its own
 * k[i]-th distance and visits its nprobe[i] lists.  Every query's result is
 * bit-identical to dade_query with that query's K and nprobe.  k, nprobe:
 * host or device [nq] (host values are checked: 1..k_max, 1..nprobe_max;
 * device values are clamped into those ranges).  ids, dists: [nq * k_max],
 * row i holding query i's k[i] results, then id -1 / +inf.  The tile schedule
 * (opts NULL or DADE_SCHED_TILE) or the row rounds (DADE_SCHED_ROUNDS) where
 * they run list-major (D > 112, delta_d of 16, 32, 64 or 128 dims, neither
 * DADE_FLAG_SEED_SPLIT nor DADE_FLAG_LEAD; DADE_EUNSUPPORTED otherwise);
 * DADE_EINVAL for other schedules.
 */
dade_status dade_query_mixed(const dade_index *ix, const float *q, int64_t nq, const int32_t *k,
                             const int32_t *nprobe, int32_t k_max, int32_t nprobe_max, float alpha, int32_t delta_d,
                             const dade_search_opts *opts, int64_t *ids, float *dists, dade_stream stream);

/* Largest nq * n_clusters one dade_probe_noalloc call accepts (16 MiB of floats). */
enum { DADE_PROBE_NOALLOC_MAX = 4194304 };

/*
 * dade_probe without any device memory allocation (the paper has no
 * counterpart; this is a library facility).  For callers that must not call
 * cudaMalloc: a serving path that must not block on or fail in the allocator
 * in the middle of a request, or a process whose device memory belongs to
 * another framework's arena.  Same inputs, outputs and results as
 * dade_probe, but q_rot and probe must be device pointers, and the query x
 * list distance matrix lives in a fixed 16 MiB array that the library holds
 * on every GPU that loads it (until exit) instead of in the index workspace.
 * nq * n_clusters above DADE_PROBE_NOALLOC_MAX is rejected with DADE_EINVAL.
 * The first call on a device looks up that array's device address (with the
 * device current), so make it before capturing a stream.  All calls share
 * the array: calls whose work can overlap on the GPU (unordered streams)
 * race and must be serialised by the caller.
 */
dade_status dade_probe_noalloc(const dade_index *ix, const float *q_rot, int64_t nq, int32_t nprobe,
                               int32_t *probe, dade_stream stream);

/*
 * Reserve workspace for searches of up to max_nq queries with up to
 * max_nprobe lists, so that later calls within these limits allocate nothing
 * (e.g. before capturing them in a CUDA graph).
 */
dade_status dade_reserve(dade_index *ix, int64_t max_nq, int32_t max_nprobe);

/*
 * eps_d (Eq. 14) and the per-increment pruning coefficients used by the scan
 * for significance alpha and step delta_d.  eps: host [d + 1], eps[dd] set for
 * every tested dd = delta_d, 2 delta_d, ... < D (others NaN).  coef: host
 * [d + 1] or NULL, coef[dd] = (1 + eps_dd)^2 * Lambda_dd / Lambda_D rounded to
 * FP32 (prune iff P_dd > coef[dd] * r^2, the squared form of the test).
 */
dade_status dade_eps_table(const dade_index *ix, float alpha, int32_t delta_d, double *eps, float *coef);

/*
 * Wait for the work queued on `stream`, then report and clear any failure
 * that the index's kernels recorded on the device since the last check
 * (DADE_ETIMEOUT from a bounded wait).  Calls with host outputs check this
 * themselves.
 */
dade_status dade_sync(const dade_index *ix, dade_stream stream);

dade_status dade_index_info(const dade_index *ix, dade_info *info);

/* Host copy of one field (see dade_field); bytes must equal the field's size. */
dade_status dade_index_export(const dade_index *ix, int32_t field, void *dst, size_t bytes);

/*
 * Host FP64 symmetric eigendecomposition used by dade_build_index
 * (Householder tridiagonalisation, then implicit symmetric QR with Wilkinson
 * shifts).  a: host [n * n] symmetric (overwritten); w: host [n] eigenvalues,
 * descending; v: host [n * n], column k = unit eigenvector of w[k].
 */
dade_status dade_host_sym_eig(double *a, int32_t n, double *w, double *v);

/*
 * HNSW* (Section 3.4; the graph of Section 4.1): greedy beam search on a
 * layer-0 graph with one DADE DCO per neighbour.  The search keeps a result
 * set R of at most ef objects and repeatedly expands the nearest object of R
 * not yet expanded: each of its neighbours not yet visited gets a DCO
 * (Algorithm 1, the Section 3.3 test) against r = the farthest distance in R
 * (+inf while R holds fewer than ef), read once per expanded object, and the
 * accepted ones enter R, which keeps its ef nearest.  The search ends when
 * every object of R is expanded or when max_visits DCOs have run; the K
 * nearest of R are the result.  Distances are FP32 sums of squares taken in
 * dimension order with every step rounded (the arithmetic of the paper's
 * scalar implementation), the test in squared form P_d > c_j r^2 with
 * c_j = (1 + eps_d)^2 Lambda_d / Lambda_D.  A structure serves one call at a
 * time (its scratch is shared by its calls).
 *
 * The graph (dade_hnsw_build): for every object the kc nearest other objects
 * by the index's FDScanning search over its nprobe nearest lists (exact when
 * nprobe = n_clusters), HNSW's neighbour heuristic (Malkov and Yashunin,
 * Algorithm 4: a candidate is kept iff it is nearer to the object than to
 * every candidate kept before it) keeping at most M, then the reverse links,
 * and over any list longer than M0 the heuristic again with cap M0.  Rows are
 * the index's rotated vectors, row-major (n * dp floats, dp = d rounded up to
 * 16), plus n * M0 int32 links.  The entry object is the one nearest the data
 * mean (smallest rotated norm, lowest id on ties).
 */
typedef struct dade_hnsw dade_hnsw;
typedef struct {
    int32_t M;                 /* links the heuristic keeps per object (default 16) */
    int32_t M0;                /* layer-0 degree cap (default 32; M <= M0 <= 32) */
    int32_t kc;                /* candidates per object (default 64; M <= kc <= 255) */
    int32_t nprobe;            /* lists of the candidate search (0: min(n_clusters, 64)) */
    int32_t reserved[4];
} dade_hnsw_build_opts;
typedef struct {
    int32_t mode;              /* DADE_MODE_DADE (default) or DADE_MODE_FD */
    int32_t n_entry;           /* entry objects per query when entry is set (1..64) */
    const int64_t *entry;      /* host or device [nq * n_entry] entry object ids (ids outside 0..n-1 are
                                  skipped); NULL: the structure's entry object */
    int64_t max_visits;        /* DCOs after which no object is expanded (0: min(n, 64 ef + 1024)) */
    const float *coef;         /* host [ceil(d / delta_d) - 1] c_j of the j-th tested d = (j + 1) delta_d;
                                  NULL: from the index's eps sample at alpha (as dade_eps_table) */
    int64_t *stats;            /* host or device [nq * 5] or NULL: DCOs run, sum of dims used, accepted,
                                  pruned (rejected before d = D), objects expanded */
    int32_t reserved[4];
} dade_hnsw_search_opts;
typedef struct {
    int64_t n;                 /* objects */
    int32_t d;                 /* dimensions */
    int32_t m0;                /* links per object */
    int64_t entry;             /* default entry object */
    int64_t device_bytes;      /* rows and links on the device */
} dade_hnsw_info;
void dade_hnsw_build_opts_default(dade_hnsw_build_opts *opts);
void dade_hnsw_search_opts_default(dade_hnsw_search_opts *opts);
/* Build over the index's own objects: base host or device [n * d] FP32, the vectors the index was built
 * on (n = the index's n; not a shard).  The index must outlive the structure.  Synchronous. */
dade_status dade_hnsw_build(const dade_index *ix, const float *base, int64_t n, const dade_hnsw_build_opts *opts,
                            dade_hnsw **out);
/* A structure over given rotated vectors x_rot (host or device [n * d] FP32) and links nbr (host or device
 * [n * m0] int32, -1 unused; 1 <= m0 <= 32), entry object `entry`.  ix (may be NULL): the index whose
 * rotation and eps sample dade_hnsw_query and a search without opts.coef use (d must match).
 * Synchronous. */
dade_status dade_hnsw_create(const dade_index *ix, const float *x_rot, int64_t n, int32_t d, const int32_t *nbr,
                             int32_t m0, int64_t entry, dade_hnsw **out);
/* Search on rotated queries q_rot (host or device [nq * d]).  1 <= k <= DADE_MAX_K, k <= ef <= 1024,
 * delta_d a multiple of 16 in [16, 1024], alpha in (0, 1) unless opts.coef is set or mode is FD.
 * ids, dists: host or device [nq * k], ascending by (squared distance, id), missing places -1 / +inf.
 * Asynchronous on `stream` for device outputs; with a host output the call returns when it is written. */
dade_status dade_hnsw_search(dade_hnsw *h, const float *q_rot, int64_t nq, int32_t k, int32_t ef, float alpha,
                             int32_t delta_d, const dade_hnsw_search_opts *opts, int64_t *ids, float *dists,
                             dade_stream stream);
/* dade_hnsw_search on raw queries q (host or device [nq * d]), rotated with the structure's index. */
dade_status dade_hnsw_query(dade_hnsw *h, const float *q, int64_t nq, int32_t k, int32_t ef, float alpha,
                            int32_t delta_d, const dade_hnsw_search_opts *opts, int64_t *ids, float *dists,
                            dade_stream stream);
dade_status dade_hnsw_info_get(const dade_hnsw *h, dade_hnsw_info *out);
/* The links, host or device [n * m0] int32.  Synchronous. */
dade_status dade_hnsw_graph(const dade_hnsw *h, int32_t *nbr);
void dade_hnsw_free(dade_hnsw *h);

/*
 * Allocation-failure injection (no counterpart in the paper; for tests of the
 * failure paths).  While a hook is set, every device allocation the library
 * makes first calls hook(bytes, user); a nonzero return makes that
 * allocation fail as a failed cudaMalloc would: the call returns DADE_ENOMEM
 * with a message naming the hook, after freeing what it had allocated.
 * NULL removes the hook.  Process-wide; set it while no call is running.
 */
typedef int (*dade_alloc_hook)(size_t bytes, void *user);
void dade_set_alloc_hook(dade_alloc_hook hook, void *user);

/* Message of the last failure on the calling thread ("" if none). */
const char *dade_last_error(void);

/* Kernels this library has launched in this process (all streams, all
 * indexes); the difference over a region counts that region's launches. */
unsigned long long dade_launch_count(void);

/*
 * Measured FP32 fused multiply-add throughput of the current GPU in TFLOP/s
 * (an FMA counts 2 FLOPs): a kernel of independent FMA chains filling every
 * SM, launched iters x 16 x 8 FMAs per thread, timed with CUDA events on
 * `stream` (best of three after a warm-up launch).  No counterpart in the
 * paper: the denominator of the arithmetic roofline of the list-major scan
 * kernels, whose staged rows are shared by many queries.  Synchronises
 * `stream`; allocates a small output buffer.
 */
dade_status dade_fp32_fma_peak(int32_t iters, double *tflops, dade_stream stream);

/* Library version string. */
const char *dade_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DADE_H */
