/*
 * ann.h -- C ABI of the GB300 graph-search library (libann.so).
 *
 * The library answers K-nearest-neighbour queries over a fixed similarity
 * graph with the best-first search of Speed-ANN (arXiv 2201.13007). The
 * problem statement it follows is Def. 1 and 2 of Sec. 2.1: given a point set
 * P of n points in d dimensions (preprocessed once into an index) and a query
 * q, return the K points of P closest to q. Closeness is the l2 distance
 * (Sec. 2.1), ranked and reported as its square; inner product (not in the
 * paper) ranks by key = -<q, x>.
 *
 * Conventions for every call:
 *   - Return value: ANN_OK (0) or a negative ann_status. On failure
 *     ann_last_error() returns a message for the calling thread.
 *   - Argument errors are detected on the host before anything is enqueued;
 *     nothing is written to the outputs then.
 *   - "device pointer" means memory of the current CUDA device (cudaMalloc,
 *     torch CUDA tensors); "host pointer" means ordinary or pinned host memory.
 *   - Streams are passed as void* holding a cudaStream_t (NULL = legacy
 *     default stream). Calls on a stream are asynchronous unless stated.
 *   - Vertex ids are int32 in the graph and int64 in results; n < 2^31.
 *   - The total order used for results is (key ascending, id ascending).
 */
#ifndef ANN_H
#define ANN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ANN_OK = 0,
    ANN_ERR_ARG = -1,     /* invalid argument (shape, range, null pointer) */
    ANN_ERR_OOM = -2,     /* device or host allocation failed */
    ANN_ERR_CUDA = -3,    /* a CUDA call failed; the message names it */
    ANN_ERR_BUSY = -4,    /* serving: no free request slot right now */
    ANN_ERR_TIMEOUT = -5, /* serving: nothing completed within the wait limit */
    ANN_ERR_STATE = -6    /* object used in a state that does not allow the call */
} ann_status;

/* Storage type of the base vectors inside the index. Reduced-precision
 * storage cuts the bytes gathered per distance; distances are always
 * accumulated in FP32. */
typedef enum {
    ANN_STORE_F32 = 0,
    ANN_STORE_BF16 = 1,
    ANN_STORE_F16 = 2,
    ANN_STORE_E4M3 = 3 /* OCP FP8 E4M3 with one FP32 scale per vector: max|x|/448 */
} ann_storage;

typedef enum { ANN_METRIC_L2 = 0, ANN_METRIC_IP = 1 } ann_metric;

/* Search modes (Sec. 4):
 *   ANN_MODE_SYNC  -- bulk-synchronous top-M expansion with the staged
 *                     schedule (Sec. 4.1, 4.2); deterministic; BFiS
 *                     (Algorithm 1) is M = 1.
 *   ANN_MODE_ASYNC -- Algorithm 3: walkers with private queues, a shared
 *                     visited map updated without ordering, and the
 *                     update-position merge test of Algorithm 2. */
typedef enum { ANN_MODE_SYNC = 0, ANN_MODE_ASYNC = 1 } ann_mode;

/* ann_index_create flags */
#define ANN_INDEX_DEVICE_INPUT 0x1 /* base and adj are device pointers */
#define ANN_INDEX_KEEP_F32 0x2     /* keep an FP32 copy of the base for re-rank */

typedef struct ann_index ann_index;

typedef struct {
    int64_t n;
    int32_t d;
    int32_t d_pad;       /* row length in elements; rows are padded with zeros to 16 bytes */
    int32_t R;           /* adjacency row length (degree cap) */
    int32_t storage;     /* ann_storage */
    int32_t metric;      /* ann_metric */
    int32_t has_f32;     /* 1 if an FP32 copy is kept for re-rank */
    int64_t entry;
    int64_t device_bytes; /* HBM held by the index */
    int64_t n_hot;        /* vertices with a neighbour group (ann_index_group_neighbors) */
} ann_index_info;

/* Per-query counters, written by the search kernels when requested. */
typedef struct {
    int64_t steps;        /* BSP steps (sync) or global steps (async) */
    int64_t expansions;   /* vertices expanded (marked checked) */
    int64_t evals;        /* distance computations, entry included */
    int64_t hash_resets;  /* visited-table resets (the table forgets, Sec. 4.4 tolerates re-visits) */
    int64_t dup_dropped;  /* candidates dropped because their id was already queued */
    int64_t merges;       /* async: merges of the private queues */
    int64_t t_start_ns;   /* device globaltimer when the query started */
    int64_t t_end_ns;     /* device globaltimer when its results were written */
} ann_query_stats;

/* Optional knobs for ann_search_ex; zero-initialise and set what is needed. */
typedef struct {
    int32_t mode;       /* ann_mode; default ANN_MODE_SYNC */
    int32_t M0;         /* initial expansion width; 0 = 1 (Algorithm 3 starts at M = 1) */
    int32_t t;          /* sync mode: M doubles every t steps; 0 = 1 (Sec. 4.2 example) */
    float R_ratio;      /* async: Algorithm 2 position ratio (the paper uses 0.8 / 0.9); 0 merges at
                         * the checker's first expansion; INFINITY merges only when every walker is idle */
    int32_t rerank;     /* 1 = recompute the final queue's keys from FP32 rows (needs has_f32) */
    int32_t threads;    /* threads per CTA: 0 = auto; sync 64..512; async 64..1024 and >= 32*M */
    int32_t hash_bits;  /* log2 slots of the per-query visited table; 0 = auto, else 8..15 */
    int32_t persistent; /* 1 = persistent grid that pulls queries from a device work counter.
                         * The index keeps one counter per stream (up to 1024 streams per
                         * index; more return ANN_ERR_STATE), so persistent searches on
                         * different streams may run at the same time; calls on one stream
                         * are ordered by the stream. A stream handle that is destroyed and
                         * handed out again names the same counter: let the old stream's
                         * work finish first. */
    /* Per-query settings (device int32 arrays of nq entries, or NULL for the
     * uniform k, L, M arguments). When given, k, L and M passed to the call
     * are the maxima over the batch, and each entry must lie in [1, max]. */
    const int32_t *k_per_query;
    const int32_t *L_per_query;
    const int32_t *M_per_query;
    ann_query_stats *stats; /* device array of nq, or NULL */
    /* Work list (device int32 array of nq entries, or NULL): the search runs
     * query order[i] for i in [0, nq); query, per-query, stats and output
     * arrays are indexed by the query number and must be large enough for
     * every number in the list. NULL runs queries 0..nq-1. */
    const int32_t *order;
    /* Sync mode only: spread each query over a thread-block cluster of this
     * many CTAs (2, 4 or 8) that share the step's work through distributed
     * shared memory (lower latency per query); 1 = one CTA per query;
     * 0 = automatic: calls of 1 to 8 queries run on clusters of 8 CTAs (4 or
     * 2 when the SMs are fewer than 8 per query) if the search is not
     * persistent, asks for no phase counters, uses visited_mode 0 or 4 and
     * the index has no neighbour groups; otherwise one CTA per query. The
     * results do not depend on the choice. A clustered search is never
     * persistent (one cluster per query). */
    int32_t cluster;
    /* Sync kernels only: device int64 array of nq x 4, or NULL. When given,
     * each query's SM clock cycles spent in its step phases are written
     * there. One-CTA kernel: [0] select (first M unchecked), [1] expand
     * (adjacency rows + visited table), [2] distance gather, [3] sort +
     * dedupe + merge. Cluster kernel (cycles of the cluster's first CTA):
     * [0] select, [1] expand + distance of its own vertices, [2] exchange
     * (cluster barrier and the copy of every CTA's survivors), [3] sort +
     * dedupe + merge. These are the Expand / Merge / Seq parts of the
     * paper's time breakdown (Fig. 14). */
    int64_t *phase_cycles;
    /* Visited set: 1 = open-addressing table of ids, exact until it is half
     * full, then reset to the queued ids; 2 = direct-mapped cache that
     * forgets a vertex when another one hashes to its slot, storing in each
     * slot only the bits of the (bijectively) hashed id that the slot index
     * does not already fix: one byte per slot while the ids need at most
     * hash_bits + 7 bits, two bytes up to hash_bits + 15, else a full id;
     * 3 = the same cache with a full 32-bit id per slot; 4 = a
     * set-associative cache: 2^hash_bits sets of one 32-bit word, each
     * holding the tags (the same split of the hashed id) of the 3 (or, for
     * ids too long for three, 2) vertices that entered the set last; a
     * fourth evicts the oldest. 2 and 3 are for the one-CTA sync kernel
     * only; clusters take 4 (each CTA holds the vertices it owns). 0 = auto
     * (one-CTA sync kernel: 4 when L >= 128, else 3; async walkers and
     * clusters: 4). No
     * form ever reports a vertex it did not see; they only forget. In sync
     * mode that changes the number of distance evaluations but never the
     * results; asynchronous walkers may also queue and expand a forgotten
     * vertex again, which changes when Algorithm 2 merges. */
    int32_t visited_mode;
    /* Sync kernels: 1 = the row of every vertex that passes the visited
     * filter is requested into L2 with one bulk prefetch
     * (cp.async.bulk.prefetch.L2) the moment it passes, so all of a step's
     * rows are in flight before the register gather reads them, and the
     * final queue's FP32 rows are requested the same way before a re-rank;
     * 2 = no prefetch; 0 = auto (1). Results never depend on it. */
    int32_t l2_prefetch;
    /* Sync kernels (one CTA or one cluster per query), distance gather:
     * lanes that share one candidate row, a power of two from 1 to 32. Each
     * lane streams its own 16-byte chunks of the row (four in flight) and the
     * team adds its partial sums with log2(team_lanes) shuffles. -1 = one
     * chunk per lane (as many lanes as the row has chunks, up to 32); 0 =
     * auto (4 lanes for rows of up to 1 KB, else 8). The FP32 partial sums
     * are added in an order that depends on it, so keys of non-integer data
     * can differ in the last bits between settings; integer-valued data
     * gives identical keys. */
    int32_t team_lanes;
    /* Async mode: the merge test of the walkers. 0 = Algorithm 2 (mean
     * update position >= L * R_ratio). 1 = stall count: each walker counts
     * its expansions since the deal that put no new candidate into the first
     * L entries of its private queue, and the checker merges when the mean
     * count over the walkers that received a non-empty deal reaches
     * `patience` (INFINITY = never early). Sec. 4.3 leaves the metric open;
     * this one measures the wasted expansions directly. */
    int32_t merge_rule;
    float patience;
    /* One-CTA sync kernel, distance gather: 1 = each warp gathers the rows of
     * the vertices it found fresh (no barrier between expand and distance);
     * 2 = the CTA's fresh vertices go into one list that all warps gather
     * (one barrier more, balanced when rows are long and few per warp); 0 =
     * auto (2). Results never depend on it. */
    int32_t gather;
} ann_search_params;

/* Build an index (Sec. 2.1: "preprocess P").
 *   base   n x d float32, row-major (host or device, see flags).
 *   adj    n x R int32, row-major, entries in [-1, n), -1 = no edge; the
 *          graph of Sec. 3.1 (stored CSR in the paper, fixed degree here).
 *   entry  the starting point P of Algorithm 1, in [0, n).
 *   storage, metric  see the enums; flags ANN_INDEX_*.
 * The library copies everything into memory it owns; the caller keeps its
 * buffers. Reduced-precision storage encodes on the device. Errors:
 * ANN_ERR_ARG for n < 1, n >= 2^31, d not in [1, 4096], R not in [1, 256],
 * entry out of range or an adjacency id out of range; ANN_ERR_OOM;
 * ANN_ERR_CUDA. Synchronous: returns when the index is ready. */
int ann_index_create(const float *base, int64_t n, int32_t d, int32_t storage, const int32_t *adj,
                     int32_t R, int64_t entry, int32_t metric, int32_t flags, ann_index **out);

/* Free everything the index owns. NULL is a no-op. The caller must not
 * destroy an index while searches on it are in flight. */
void ann_index_destroy(ann_index *index);

/* Shape and storage of an index. */
int ann_index_get_info(const ann_index *index, ann_index_info *info);

/* Neighbour grouping (Sec. 4.4, cache-friendly neighbour grouping, in its
 * degree-centric form): for the round(hot_fraction * n) vertices with the
 * most in-edges (ties: the smaller id), store a copy of their R neighbours'
 * stored rows contiguously, in adjacency order, after the n base rows (and
 * scales). When the one-CTA sync kernel expands such a vertex it reads the
 * fresh neighbours' vectors from that block instead of from R scattered
 * rows; prefetch = 0 asks L2 for the whole block with one bulk prefetch when
 * the vertex is expanded, prefetch = 1 asks only for the fresh rows, as for
 * other vertices. The copies hold the same values, so results do not
 * change. Vertex ids are not relabelled (they fix the (key, id) order of
 * every result). hot_fraction in [0, 0.05]; 0 removes the grouping. Costs
 * hot_fraction * n * R extra rows of HBM. Synchronous; no search may be in
 * flight on the index. Errors: ANN_ERR_ARG, ANN_ERR_STATE (wrong device),
 * ANN_ERR_OOM, ANN_ERR_CUDA. */
int ann_index_group_neighbors(ann_index *index, float hot_fraction, int32_t prefetch);

/* Exact k nearest base rows of every query row by a brute-force scan
 * (Def. 1 of Sec. 2.1 over BF16 data), for building the similarity graph
 * the search runs on; the paper assumes the graph exists (Sec. 2.2), and its
 * k-NN candidate lists are these neighbours. The n x nq distance matrix is
 * never stored: tensor-core tiles of it are filtered into per-row top-64
 * lists in shared memory.
 *   base       device, n x d BF16 bit patterns, row-major, 16-byte aligned.
 *   queries    device, nq x d BF16 bit patterns, row-major, 16-byte aligned
 *              (may be a slice of base).
 *   d          32, 64, 96 or 128.
 *   self_offset -1, or the base row of query 0: query i is then base row
 *              self_offset + i and is left out of its own result.
 *   metric     ann_metric; keys are squared l2 or -<q, x>, products exact
 *              in FP32 and sums in FP32.
 *   k          1..64 results per query.
 *   out_ids    device int32 nq x k, out_dists device float nq x k, ascending
 *              by (key, id); slots beyond the available rows hold (-1, +inf).
 * Synchronous (the call waits for stream). Errors: ANN_ERR_ARG (shape,
 * alignment, range), ANN_ERR_OOM, ANN_ERR_CUDA. Work: n * nq * d
 * multiply-adds on the tensor cores, plus 256 threads per 128 queries. */
int ann_knn_bf16(const void *base, int64_t n, int32_t d, const void *queries, int64_t nq, int64_t self_offset,
                 int32_t metric, int32_t k, int32_t *out_ids, float *out_dists, void *stream);

/* Search nq queries (Algorithm 1 / Sec. 4.1-4.2 top-M with M doubling from 1,
 * one CTA per query).
 *   queries    device, nq x d float32 row-major.
 *   k          results per query (the paper's K), 1 <= k <= L.
 *   L          candidate-queue capacity of Algorithm 1, 1 <= L <= 2048.
 *   M          maximum expansion width (the paper's M, capped by T), 1..64
 *              (async mode: the number of walkers T, 1..32).
 *   out_ids    device int64 nq x k; out_dists device float nq x k (squared
 *              l2, or -<q,x>). Slots beyond the reachable set hold (-1, +inf).
 * Asynchronous on stream; argument errors return before anything is queued.
 * nq = 0 is a no-op. Equivalent to ann_search_ex with default params. */
int ann_search(const ann_index *index, const float *queries, int64_t nq, int32_t k, int32_t L,
               int32_t M, int64_t *out_ids, float *out_dists, void *stream);

/* ann_search with the knobs of ann_search_params (mode, schedule, re-rank,
 * per-query k/L/M, counters). params may be NULL. */
int ann_search_ex(const ann_index *index, const float *queries, int64_t nq, int32_t k, int32_t L,
                  int32_t M, int64_t *out_ids, float *out_dists, const ann_search_params *params,
                  void *stream);

/* Launch configuration ann_search_ex would use for these arguments,
 * without launching anything (argument errors as in ann_search_ex). */
typedef struct {
    int32_t threads;      /* threads per CTA */
    int32_t smem_bytes;   /* dynamic shared memory per CTA */
    int32_t grid;         /* CTAs launched */
    int32_t hash_bits;    /* log2 slots of the visited table */
    int32_t cluster;      /* CTAs per query */
    int32_t mode;         /* ann_mode */
    int32_t visited_slot_bytes; /* bytes per visited-set slot: 1 or 2 (tags), 4 (ids or a set word) */
    int32_t visited_ways;       /* set-associative visited cache: tags per set word (2 or 3); 0 = other form */
} ann_launch_info;

int ann_search_describe(const ann_index *index, int64_t nq, int32_t k, int32_t L, int32_t M,
                        const ann_search_params *params, ann_launch_info *out);

/* The same search from HOST buffers: copies the queries to the device,
 * searches, copies the results back and synchronises the stream before it
 * returns. queries host nq x d float32; out_ids / out_dists host nq x k.
 * Pinned host memory keeps the copies asynchronous to the CPU. The library
 * keeps device staging buffers per index, grown on demand (the index must
 * not be used by two host-buffer calls at once). params may be NULL; its
 * per-query arrays, if any, must be device pointers. */
int ann_search_host(ann_index *index, const float *queries, int64_t nq, int32_t k, int32_t L,
                    int32_t M, int64_t *out_ids, float *out_dists, const ann_search_params *params,
                    void *stream);

/* Size of the static device array behind ann_search_host_noalloc. */
#define ANN_NOALLOC_SCRATCH_BYTES (16u << 20)

/* ann_search_host for callers that cannot allocate device memory when they
 * search: a process whose device memory is reserved up front by another
 * framework's caching allocator (so a cudaMalloc here would fail or fragment
 * its pool), or a latency-critical thread that must not enter the CUDA
 * allocator, which can block on the device. The paper has no counterpart.
 *   Arguments, layout and results are those of ann_search_host (host
 *   buffers in and out, params may be NULL; the search always runs as a
 *   persistent grid with one CTA per query). params->cluster must be 0 or 1
 *   (ANN_ERR_ARG otherwise). The call allocates nothing: its device scratch
 *   (the persistent grid's work counter and device copies of the queries
 *   and of the results) lives in one static device array of
 *   ANN_NOALLOC_SCRATCH_BYTES (16 MiB) that every GPU which loads the
 *   library holds until the process exits.
 *   A batch needing more than that (256 + nq*d*4 + nq*k*12 bytes, each part
 *   rounded up to 256) is rejected with ANN_ERR_ARG and a message giving the
 *   size and the limit.
 *   The first call on a device resolves the array's address on that device
 *   (this may load the module), so make that first call before any stream
 *   capture.
 *   All calls share the one array, which keeps the last call's contents;
 *   calls that overlap on the GPU (other streams, other threads) race on it
 *   and must be serialised by the caller. Copies from and to the caller's
 *   host buffers and synchronises the stream before it returns. */
int ann_search_host_noalloc(const ann_index *index, const float *queries, int64_t nq, int32_t k, int32_t L,
                            int32_t M, int64_t *out_ids, float *out_dists, const ann_search_params *params,
                            void *stream);

/* ------------------------------------------------------------ batching
 * A planned batch of queries with uneven k, L, M (no counterpart in the
 * paper, which runs one query at a time). Queries are grouped into buckets
 * by L; each bucket is one persistent grid, sized for the bucket's largest L
 * and M, that pulls its queries longest-first from a device work list. The
 * buckets run concurrently on the plan's own streams, forked from and joined
 * back into the caller's stream, so a whole ann_batch_search can be captured
 * into a CUDA graph (it allocates nothing and never synchronises). */

typedef struct {
    int32_t L_max;      /* the bucket takes queries with L <= L_max (after smaller buckets) */
    int32_t threads;    /* launch config for the bucket; 0 = the ann_search_ex default */
    int32_t hash_bits;
} ann_bucket_config;

typedef struct ann_batch ann_batch;

/* Plan nq queries. k, L, M are HOST int32 arrays of nq entries (each with
 * 1 <= k <= L <= 2048, 1 <= M <= 64). buckets: n_buckets configs in
 * ascending L_max, or NULL for the ladder 32, 64, 128, 256, 512, 1024, 2048
 * with default launch configs. params supplies mode, schedule, re-rank and an
 * optional stats array (its per-query arrays and order must be NULL). The
 * plan keeps device copies of k, L, M and of the work lists; the index must
 * outlive it. Errors: ANN_ERR_ARG, ANN_ERR_OOM, ANN_ERR_CUDA. */
int ann_batch_create(const ann_index *index, int64_t nq, const int32_t *k, const int32_t *L, const int32_t *M,
                     const ann_bucket_config *buckets, int32_t n_buckets, const ann_search_params *params,
                     ann_batch **out);

/* Run the planned batch on stream. queries: device nq x d; out_ids / out_dists:
 * device nq x k_max with k_max = the largest k in the plan (entries past a
 * query's own k hold -1 / +inf). Asynchronous. Calls on one plan must not
 * overlap on the GPU (the plan's work counters are reset by each call). */
int ann_batch_search(ann_batch *batch, const float *queries, int64_t *out_ids, float *out_dists, void *stream);

/* Number of non-empty buckets and the largest k of a plan. */
int ann_batch_info(const ann_batch *batch, int32_t *n_buckets, int32_t *k_max);

/* Free a plan (after its searches have finished). NULL is a no-op. */
void ann_batch_destroy(ann_batch *batch);

/* Message of the last failing call on this thread ("" if none). */
const char *ann_last_error(void);

/* ---------------------------------------------------------------- serving
 * Continuous batching (no counterpart in the paper, which processes one
 * query at a time, Sec. 5). Requests are submitted one at a time from the
 * host and admitted to the GPU as request groups free up. A group is a
 * block of device-resident request state (queries, per-request k / L / M,
 * results, counters) for max_batch requests; `streams` groups exist, so at
 * most streams * max_batch requests are on the device at once, and the
 * device memory they take is the admission budget. The library's scheduler
 * thread fills any free group with the waiting requests and launches it on
 * that group's own stream, so requests that arrive while others are on the
 * GPU run alongside them. In sync mode each result is exactly the result of
 * a single ann_search_ex of that query with the same k, L, M and params. */

typedef struct {
    int32_t slots;          /* requests accepted and not yet collected; 0 = 4 * streams * max_batch */
    int32_t max_batch;      /* requests per launch (one group); 0 = 1024 */
    int32_t streams;        /* groups, i.e. launches in flight at once; 0 = 4 */
    int32_t max_k;          /* per-request limits; 0 = 100 / 1024 / 32 */
    int32_t max_L;
    int32_t max_M;
    int32_t mode;           /* ann_mode for every request */
    int32_t rerank;         /* as in ann_search_params */
    int64_t scratch_bytes;  /* cap on the device bytes of all groups; 0 = no cap.
                             * streams is lowered until the groups fit. */
} ann_serve_config;

typedef struct ann_server ann_server;

typedef struct {
    uint64_t tag;             /* the caller's tag from ann_serve_submit */
    int32_t k;                /* valid entries in ids / dists */
    int32_t status;           /* ANN_OK or the request's error */
    double latency_us;        /* submit to completion, host clock */
    double device_us;         /* the query's own time on the device */
    int64_t device_start_ns;  /* device globaltimer at the query's start and end */
    int64_t device_end_ns;
} ann_result;

/* Create a server over an index (the index must outlive the server). The
 * index's device must be current. Errors: ANN_ERR_ARG for limits outside
 * those of ann_search_ex, ANN_ERR_OOM, ANN_ERR_CUDA. */
int ann_serve_create(const ann_index *index, const ann_serve_config *cfg, ann_server **out);

/* Finish every accepted request, stop the scheduler and free everything.
 * Results not yet collected are dropped. NULL is a no-op. */
void ann_serve_destroy(ann_server *server);

/* Submit one query (host pointer to d float32, copied before return) with
 * its own k, L, M and a caller tag. Never blocks: returns ANN_ERR_BUSY when
 * `slots` requests are already accepted and not yet collected, ANN_ERR_ARG
 * for k, L, M outside the config (or k > L). Thread safe. */
int ann_serve_submit(ann_server *server, const float *query, int32_t k, int32_t L, int32_t M,
                     uint64_t tag);

/* Collect up to max completed requests (completion order). results[i]
 * describes request i; its ids / dists are written to
 * out_ids + i * cfg.max_k and out_dists + i * cfg.max_k (host; entries past
 * results[i].k are padded with -1 / +inf). Waits at most timeout_us
 * microseconds for the first completion and returns the number collected
 * (>= 1), or ANN_ERR_TIMEOUT when nothing completed in time. Thread safe. */
int ann_serve_poll(ann_server *server, ann_result *results, int64_t *out_ids, float *out_dists,
                   int32_t max, int32_t timeout_us);

/* Drive a server with a request trace from native threads (a load
 * generator without the caller's per-request overhead): request i asks for
 * row qi[i] of the host array queries (n_queries x d float32) with k[i],
 * L[i], M[i], and is submitted arrival_us[i] microseconds after the call
 * starts (host steady clock; arrival_us non-decreasing, or NULL to submit
 * every request as fast as the server accepts it). A submission that finds
 * every slot taken is retried until one frees. The calling thread collects
 * the completions meanwhile. Outputs, per request (host arrays of nreq):
 * latency_us (submit to completion, as ann_result.latency_us), device_us,
 * and status; *wall_us is the time from the start to the last completion;
 * *busy_retries (may be NULL) counts the retried submissions. The server
 * must have no other client during the call. Synchronous. Errors:
 * ANN_ERR_ARG; ANN_ERR_TIMEOUT if the trace is not complete 60 s after its
 * last arrival (requests still in flight are then collected by later
 * ann_serve_poll calls). The paper has no counterpart (it measures one
 * query at a time). */
int ann_serve_replay(ann_server *server, const float *queries, int64_t n_queries, const int64_t *qi,
                     const int32_t *k, const int32_t *L, const int32_t *M, const double *arrival_us,
                     int64_t nreq, double *latency_us, double *device_us, int32_t *status, double *wall_us,
                     int64_t *busy_retries);

#ifdef __cplusplus
}
#endif

#endif /* ANN_H */
