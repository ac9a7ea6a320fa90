/*
 * pdx.h -- C ABI of the GB300 (sm_103a) PDX vector-search library.
 *
 * The library stores vectors in the PDX layout (Sec. 3 of "PDX: A Data Layout
 * for Vector Similarity Search", Kuffo, Krippner, Boncz, SIGMOD'25): vectors
 * are grouped in blocks of 64 and, inside a block, stored dimension by
 * dimension (element (vector t, dimension j) of block b at
 * data[(b*D + j)*64 + t]). Searches run the PDXearch framework (Sec. 4: START,
 * WARMUP, PRUNE phases with doubling fetch steps) with the PDX-BOND (Sec. 5),
 * ADSampling or BSA (Sec. 2.3) pruning predicates, and return the k nearest
 * neighbours defined in Sec. 2.1.
 *
 * Conventions shared by every call:
 *  - All functions are extern "C" and never throw. A non-OK status leaves a
 *    thread-local message readable through pdx_last_error().
 *  - Pointers to vectors, queries and outputs may be host or device memory of
 *    the current device; the library tells them apart with
 *    cudaPointerGetAttributes. The caller owns them; the library copies what
 *    it needs and keeps no reference after the call returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). With device outputs a search is asynchronous on `stream`; with
 *    host outputs (or a non-NULL stats_out) it synchronises `stream` before
 *    returning.
 *  - Vectors and queries are row-major float32: x[i*d + j], q[i*d + j].
 *  - Outputs are row-major [nq][k], best first: L2 and L1 ascending, IP
 *    descending; equal distances are ordered by the lower vector id. A row
 *    with fewer than k results is padded with id -1 and distance +inf
 *    (-inf for IP).
 *  - Search scratch memory is taken from the stream-ordered allocator
 *    (cudaMallocAsync) and released on `stream` before the call returns, so
 *    concurrent searches on the same index from different threads/streams are
 *    safe. An index must not be freed while a search on it is in flight.
 *  - Limits: 1 <= d <= 4096, 1 <= k <= 1024, n < 2^31.
 */
#ifndef PDX_H_
#define PDX_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pdx_index pdx_index; /* opaque; owns all of its device memory */
typedef struct pdx_mlp pdx_mlp;     /* opaque order-proposal network (see pdx_mlp_create) */

typedef enum pdx_status {
    PDX_OK = 0,
    PDX_ERR_ARG = 1,          /* invalid argument; outputs untouched          */
    PDX_ERR_OOM = 2,          /* device allocation failed                     */
    PDX_ERR_CUDA = 3,         /* a CUDA call failed                           */
    PDX_ERR_TIMEOUT = 4,      /* a bounded device wait ran out                */
    PDX_ERR_UNSUPPORTED = 5   /* valid request the library does not implement */
} pdx_status;

/* Sec. 2.1: squared Euclidean distance, inner product (similarity, larger is
 * better), Manhattan distance; Listing 1 gives the three PDX kernels. */
typedef enum pdx_metric { PDX_L2 = 0, PDX_IP = 1, PDX_L1 = 2 } pdx_metric;

/* Storage type of the PDX blocks. BF16 / FP8-E4M3 storage keeps an FP32 copy
 * for the final rerank; FP32 accumulation throughout. */
typedef enum pdx_dtype { PDX_F32 = 0, PDX_BF16 = 1, PDX_FP8_E4M3 = 2 } pdx_dtype;

/* Pruning predicates (Sec. 2.3 and Sec. 5). NONE is the PDX linear scan. */
typedef enum pdx_pruner {
    PDX_PRUNE_NONE = 0,
    PDX_PRUNE_BOND = 1,        /* exact: partial distance > tau              */
    PDX_PRUNE_ADSAMPLING = 2,  /* approximate: hypothesis test, eps0         */
    PDX_PRUNE_BSA = 3,         /* approximate: error quantile, multiplier m  */
    PDX_PRUNE_ADS_BOND = 4,    /* approximate: ADSampling on a rotated index with
                                  PDX-BOND's query-aware visit order (the fusion
                                  Sec. 8 proposes as future work). Dimensions are
                                  visited by distance to the probed bucket's means
                                  (zones of zone_dims); after d of them a vector is
                                  pruned when partial > tau (PDX-BOND, exact) or
                                  partial > tau * F_q(d) * (1 + eps0/sqrt(d))^2,
                                  where F_q(d) is the visited share of the expected
                                  distance sum_j (q_j - mu_j)^2 + var_j over the
                                  bucket (mu, var: the bucket's means and
                                  variances). With storage order and equal
                                  expected terms it is ADSampling's test.       */
    PDX_PRUNE_CS_IP = 5        /* exact: inner product with any vector norms.
                                  Partial inner products are not monotone, so
                                  PDX-BOND's test does not apply to them; after d
                                  dimensions in storage order the unvisited part
                                  q_r . x_r is at most ||q_r|| ||x_r||
                                  (Cauchy-Schwarz, the exact bound BSA uses for L2
                                  in Sec. 2.3), and a vector is pruned when
                                  -(partial inner product) - ||q_r|| ||x_r|| > tau,
                                  tau the k-th best -q.x so far, minus a rounding
                                  margin of D * 2^-23 (||q_r|| ||x_r|| + ||q|| ||x||).
                                  Exact search over an index built with
                                  cs_first_step (its stored norms fix the fetch
                                  schedule: the search's first_step is set to it) */
} pdx_pruner;

/* Order in which PDX-BOND visits dimensions (Sec. 5, Fig. 6). */
typedef enum pdx_order {
    PDX_ORDER_DIST_TO_MEANS = 0, /* by |q_j - mu_j| of the block, descending */
    PDX_ORDER_DECREASING = 1,    /* by q_j, descending (BOND's order)        */
    PDX_ORDER_SEQUENTIAL = 2,    /* storage order                            */
    PDX_ORDER_LEARNED = 3        /* scores of an order-proposal network      */
} pdx_order;

/* Whose means the distance-to-means order uses (Sec. 5 speaks of the block's
 * statistics; the Fig. 6 caption of the collection's). Either keeps PDX-BOND
 * exact: only the amount of pruning depends on the order. */
typedef enum pdx_means_scope {
    PDX_MEANS_BLOCK = 0,       /* per PDXearch block (partition / bucket)    */
    PDX_MEANS_COLLECTION = 1,  /* of the whole collection                    */
    PDX_MEANS_AUTO = 2         /* collection for exact search (its partitions
                                  are arbitrary id ranges), block for IVF
                                  (its buckets are clusters)                 */
} pdx_means_scope;

/*
 * Engines of the unpruned exact search (pruner PDX_PRUNE_NONE).
 * SCAN   -- the PDX scan of Sec. 3/4 without a predicate: every dimension of
 *           every vector, accumulated lane by lane on the CUDA cores.
 * TENSOR -- the distance decomposition ||q||^2 + ||x||^2 - 2 q.x of Sec. 2.1
 *           with q.x from a TF32 tensor-core GEMM over query batches
 *           (tcgen05, FP32 accumulation). Every pair gets an estimate and a
 *           proven error bound; vectors whose lower bound is within the k-th
 *           smallest upper bound are reranked in FP32 from the row-major
 *           copy, so results equal the SCAN engine's (up to ties within
 *           FP32 rounding). Needs an exact index built with dense_rows, L2
 *           or IP, d a multiple of 4, k <= 64.
 * AUTO   -- TENSOR when those conditions hold and the product is large
 *           enough to pay for its fixed cost (nq * n * d >= 2^32), else SCAN.
 */
typedef enum pdx_engine {
    PDX_ENGINE_AUTO = 0,
    PDX_ENGINE_SCAN = 1,
    PDX_ENGINE_TENSOR = 2
} pdx_engine;

/*
 * Storage layouts of the linear scan (pruner PDX_PRUNE_NONE, engine SCAN),
 * for comparing layouts on one workload (Sec. 3 Fig. 3, the kernel study of
 * Sec. 6.2 / Table 3, N-ary + gather and DSM in Sec. 7). Every layout gives
 * the same exact results.
 * PDX          the index's PDX blocks (the default scan path)
 * PDX_KERNEL   the PDX blocks through the same minimal kernel the other
 *              layouts use (no phases, no threshold sharing)
 * NARY         row-major vectors (keep_rows): a warp reduces each vector's
 *              partial sums across its lanes
 * NARY_GATHER  row-major vectors staged into shared memory as 64-vector x
 *              32-dimension tiles, transposed on the fly, then the PDX kernel
 * DSM          the whole collection dimension-major (keep_dsm)
 * The layout kernels need FP32 storage, an exact index, k <= 256 and (N-ary
 * forms) d a multiple of 4; otherwise the search returns PDX_ERR_UNSUPPORTED.
 */
typedef enum pdx_layout {
    PDX_LAYOUT_PDX = 0,
    PDX_LAYOUT_PDX_KERNEL = 1,
    PDX_LAYOUT_NARY = 2,
    PDX_LAYOUT_NARY_GATHER = 3,
    PDX_LAYOUT_DSM = 4
} pdx_layout;

typedef struct pdx_build_opts {
    uint32_t struct_size;      /* = sizeof(pdx_build_opts)                                */
    pdx_metric metric;         /* metric the index will be searched with                   */
    pdx_dtype storage;         /* block storage type. BF16 / FP8_E4M3 blocks are scanned with
                                  a lower bound widened by the per-element quantisation error,
                                  and survivors are reranked from an FP32 copy of the vectors
                                  that the index keeps (n*d*4 bytes); L2 and unit-norm IP  */
    uint32_t partition_size;   /* exact search: at most this many vectors per PDXearch
                                  block, equal horizontal partitions (Sec. 6.6; 10000)    */
    int32_t keep_rows;         /* keep the vectors row-major in FP32 (n*d*4 bytes, default
                                  1). BF16/FP8 storage always keeps them: they are its
                                  rerank source. With FP32 storage the scan uses them to
                                  finish PRUNE phases that start with at most 8 survivors
                                  (exact distances from contiguous rows instead of one
                                  memory sector per value of the dimension-major block). */
    int32_t dense_rows;        /* keep, for the tensor-core dense engine, the vectors
                                  row-major in FP32 (the rerank source), a copy rounded to
                                  TF32 (the GEMM operand) and per-row norms: n*(2d+4)*4
                                  bytes. Low-precision storage keeps the FP32 rows anyway
                                  and adds n*(d+4)*4 bytes (default 0)                     */
    int32_t keep_dsm;          /* also keep the collection fully dimension-major (DSM: d
                                  columns of ceil(n/64)*64 floats) for the PDX_LAYOUT_DSM
                                  scan (default 0)                                          */
    int32_t start_clusters;    /* exact indexes: centroids that seed START (Sec. 4). The build
                                  runs k-means over a sample and keeps, per centroid, the 64
                                  vectors nearest to it; a pruned L2 search then takes its
                                  initial threshold from exact distances to the members of
                                  the query's 2 nearest centroids (more for k > 64: enough
                                  for 2k members, at most 16; real vectors near the query)
                                  instead of from the first start_vectors stored vectors. 0 = automatic (n/4096 centroids, at most 1024,
                                  for n >= 65536; none below), -1 = none                  */
    int32_t cs_first_step;     /* inner-product indexes: store, for the Cauchy-Schwarz bound
                                  of PDX_PRUNE_CS_IP, every vector's norm and the norms of
                                  its unvisited dimensions at the check points of the fetch
                                  schedule that starts with this step (check points after
                                  s, 3s, 7s, ... dimensions): 4 * (checks + 1) bytes per
                                  vector. 0 = none (default); a non-zero value needs
                                  metric PDX_IP and FP32 storage                           */
} pdx_build_opts;

typedef struct pdx_ivf_opts {
    uint32_t struct_size;      /* = sizeof(pdx_ivf_opts)                                   */
    pdx_build_opts base;       /* metric / storage; partition_size is ignored             */
    uint32_t nlist;            /* number of IVF buckets (k-means centroids)               */
    uint32_t kmeans_iters;     /* Lloyd iterations on the GPU                              */
    uint32_t kmeans_sample;    /* vectors used to train (0 = all)                         */
    uint64_t seed;             /* picks the initial centroids when none are given          */
    pdx_pruner transform;      /* ADSAMPLING: random orthogonal rotation; BSA: PCA projection */
    const float *rotation;     /* ADSAMPLING, optional: the caller's d*d orthogonal matrix,
                                  row-major (host or device, caller-owned); the stored and
                                  query vectors become rotation * v. NULL: the library draws
                                  its own from rotation_seed (below).                      */
    const float *init_centroids; /* optional nlist*d initial centroids (host or device)   */
    uint64_t rotation_seed;    /* ADSAMPLING without `rotation`: seed of the random
                                  orthogonal matrix (Sec. 2.3). The library fills a d*d
                                  matrix with standard normal values (splitmix64 counter
                                  stream, Box-Muller), takes its QR factorisation in FP64
                                  (Householder) and keeps Q with every column's sign set
                                  so that R's diagonal is positive: a Haar-distributed
                                  orthogonal matrix. Same seed, same matrix.               */
} pdx_ivf_opts;

typedef struct pdx_search_stats {
    uint64_t values_visited;   /* sum over (query, vector) of dimensions accumulated by the
                                  PDXearch scan (Sec. 2.2: pruning power = 1 - this / (nq*n*D)) */
    uint64_t vectors_scanned;  /* (query, vector) pairs touched by the scan                   */
    uint64_t vectors_pruned;   /* pairs discarded before their last dimension                 */
    uint64_t prune_phase_blocks; /* (query, 64-vector block) pairs that reached PRUNE         */
    uint64_t candidates;       /* full distances offered to the top-k lists                   */
    uint64_t work_items;       /* non-empty (query, block-group) work items                   */
    uint64_t start_values;     /* values computed by the START scan (exact search)            */
    uint64_t bytes_logical;    /* (values_visited + start_values) * element size; filled only
                                  in stats_out                                               */
    uint64_t dense_fallbacks;  /* tensor-core engine: queries whose candidates overflowed their
                                  buffer (or whose GEMM gave up on a wait) and were answered
                                  by a plain FP32 scan instead                              */
    uint64_t phase_ns[5];      /* device time of each phase of the search in nanoseconds, from
                                  CUDA events on `stream` (the breakdown of Table 6); filled
                                  only in stats_out:
                                  [0] query preprocessing: ADSampling/BSA transform, visit
                                      orders, order-network inference
                                  [1] finding the nearest IVF buckets (0 for exact search)
                                  [2] START: the initial thresholds (exact: start clusters or
                                      the first start_vectors; IVF: the nearest bucket's scan,
                                      unless a large batch runs it first inside phase [3])
                                  [3] WARMUP/PRUNE: the PDXearch scan (or the tensor engine)
                                  [4] merge of the per-item lists, canonical distances, output */
    uint64_t reserved[2];
} pdx_search_stats;

typedef struct pdx_search_opts {
    uint32_t struct_size;      /* = sizeof(pdx_search_opts)                                */
    pdx_pruner pruner;         /* default BOND                                             */
    pdx_order order;           /* PDX-BOND visit order (default DIST_TO_MEANS)             */
    uint32_t zone_dims;        /* dimension-zone width (Sec. 5); 1 = per dimension; 0 = 1
                                  with collection means, 8 with block means               */
    float selection_threshold; /* switch WARMUP -> PRUNE below this fraction (0.20)        */
    float eps0;                /* ADSampling error bound (2.1)                             */
    float bsa_m;               /* BSA multiplier m                                         */
    uint32_t first_step;       /* first fetch step in dimensions, then doubling (default 4;
                                  the paper's CPU setting is 2). BSA searches always use the
                                  schedule their index stored residual norms for (4).      */
    uint32_t start_vectors;    /* exact search: vectors of the START scan (default 1024; 0 = one block) */
    uint32_t blocks_per_item;  /* 64-vector blocks per GPU work item (0 = automatic)       */
    pdx_search_stats *stats_out; /* optional host pointer; filled after the search (the call
                                  then synchronises `stream`)                               */
    pdx_search_stats *stats_device; /* optional device pointer: the kernels add their counters
                                  to its first seven fields and dense_fallbacks asynchronously
                                  (caller zeroes it; bytes_logical is not written)           */
    void *scan_event_start;    /* optional cudaEvent_t recorded on `stream` just before the
                                  PDXearch scan kernel                                        */
    void *scan_event_stop;     /* optional cudaEvent_t recorded just after it                 */
    pdx_means_scope means_scope; /* distance-to-means order: block or collection means (AUTO) */
    uint32_t ctas_per_sm;      /* resident scan CTAs per SM (0 = 4 when four CTAs' shared
                                  memory leaves 32 KB for L1, else 3). The shared-memory
                                  carveout is sized for exactly this many, and the rest of
                                  each SM's on-chip memory serves as L1 for the loads in
                                  flight.                                                  */
    pdx_mlp *mlp;              /* PDX_ORDER_LEARNED: the network (exact indexes)           */
    const float *mlp_centroids;/* PDX_ORDER_LEARNED: device [mlp_ncentroids][d]; each query
                                  is paired with its nearest one as the network input      */
    int32_t mlp_ncentroids;
    pdx_engine engine;         /* unpruned exact search: PDX scan or tensor-core GEMM (AUTO) */
    const float *tau_init;     /* optional [nq] initial thresholds (host or device): each
                                  query's search starts from min(tau_init[i], what START
                                  finds). For an exact result each value must be at least
                                  the query's true k-th distance (e.g. the k-th distance of
                                  k real vectors); a smaller value makes the result the
                                  best vectors within it, padded. In the metric the scan
                                  ranks by (L2 or L1; unit-norm IP is searched as L2)     */
    int32_t tau_fixed;         /* nonzero (with tau_init): no START, and the thresholds never
                                  tighten during the search, so which vectors are pruned
                                  depends only on tau_init and the predicate, not on the
                                  order in which warps finish. Meant for reproducible prune
                                  counts (tests against a sequential implementation).    */
    pdx_layout layout;         /* unpruned exact search on the SCAN engine: which storage
                                  layout the linear scan reads (default PDX)               */
    uint64_t *finished_log;    /* optional device array (a check of exactness, not for
                                  speed): the PDXearch scan appends (query << 32) | id for
                                  every vector it carries through all D dimensions (it was
                                  pruned by no test), in no particular order. A pruned
                                  exact search is exact iff every query's true top-k is
                                  among its entries. FP32 blocks with PDX_PRUNE_BOND or
                                  PDX_PRUNE_CS_IP only (else PDX_ERR_UNSUPPORTED); the
                                  logging scan is a separate kernel instance, so searches
                                  without a log run unchanged. NULL (default): no log     */
    unsigned long long *finished_count; /* device counter the scan adds to (the caller zeroes
                                  it); entries beyond finished_cap are counted, not stored */
    uint64_t finished_cap;     /* capacity of finished_log in entries                      */
} pdx_search_opts;

typedef struct pdx_index_info {
    int64_t n;                 /* vectors                                                  */
    int32_t d;                 /* dimensions                                               */
    int32_t nparts;            /* PDXearch blocks: partitions (exact) or buckets (IVF)     */
    int64_t nblocks;           /* 64-vector storage blocks                                 */
    pdx_metric metric;
    pdx_dtype storage;
    int32_t is_ivf;
    int32_t unit_norm;         /* every stored vector has norm 1 (within 1e-5)             */
    uint64_t device_bytes;     /* device memory owned by the index                         */
} pdx_index_info;

/* Internal arrays that pdx_index_copy_out can return (for inspection/tests). */
typedef enum pdx_array {
    PDX_ARRAY_BLOCKS = 0,      /* float32 [nblocks][d][64] PDX storage (zero padded; F32)  */
    PDX_ARRAY_IDS = 1,         /* int32 [nblocks*64] vector id per slot, -1 = padding      */
    PDX_ARRAY_PART_BLOCKS = 2, /* int32 [nparts+1] first storage block of each part        */
    PDX_ARRAY_MEANS = 3,       /* float32 [nparts][d] per-part dimension means (Sec. 3)    */
    PDX_ARRAY_CENTROIDS = 4,   /* float32 [nparts][d] IVF centroids (transformed space)    */
    PDX_ARRAY_ASSIGN = 5,      /* int32 [n] IVF bucket of each vector                      */
    PDX_ARRAY_ROTATION = 6,    /* float32 [d][d] IVF transform applied to vectors/queries  */
    PDX_ARRAY_VARIANCES = 7,   /* float32 [d] BSA: variance of each projected dimension    */
    PDX_ARRAY_BLOCKS_LP = 8,   /* bf16 / fp8-e4m3 bits [nblocks][d][64] (storage != F32)   */
    PDX_ARRAY_SCALES = 9,      /* float32 [d] FP8 storage: per-dimension scale             */
    PDX_ARRAY_ROWS = 10        /* float32 [n][d] row-major vectors by id (keep_rows); for a
                                  rotated or projected IVF index the original vectors     */
} pdx_array;

/* Fill an options struct with the defaults named above. */
void pdx_default_build_opts(pdx_build_opts *opts);
void pdx_default_ivf_opts(pdx_ivf_opts *opts);
void pdx_default_search_opts(pdx_search_opts *opts);

/*
 * pdx_build_layout -- exact-search index (Sec. 3, Sec. 6.6).
 * Splits the n vectors x[n][d] (row-major float32, host or device) into
 * ceil(n / partition_size) equal horizontal partitions in id order, stores
 * each partition as consecutive 64-vector PDX blocks (its last block zero
 * padded) and records per-partition dimension means (block metadata, Sec. 3).
 * opts may be NULL (defaults). On success *out owns a new index; on failure
 * *out is set to NULL. Errors: PDX_ERR_ARG (NULL pointers, n < 1, d outside
 * [1,4096], bad opts), PDX_ERR_OOM, PDX_ERR_CUDA.
 */
pdx_status pdx_build_layout(const float *x, int64_t n, int32_t d, const pdx_build_opts *opts,
                            void *stream, pdx_index **out);

/*
 * pdx_ivf_build -- IVF index whose buckets are PDX blocks (Sec. 2.1, Fig. 2).
 * Optionally transforms the vectors first (ADSampling: a random orthogonal
 * rotation, the caller's or one drawn from rotation_seed; BSA: PCA projection
 * computed here), runs
 * kmeans_iters Lloyd iterations on the GPU from init_centroids (or from
 * nlist vectors picked with `seed`), assigns every vector to its nearest
 * centroid (ties: lower bucket id), and lays each bucket out as PDX blocks.
 * A transformed index keeps the original vectors row-major (keep_rows) and
 * reports every distance from them and the untransformed query, so its
 * distances carry no rounding of the transform.
 * Errors as pdx_build_layout, plus PDX_ERR_ARG for nlist outside [1, n].
 */
pdx_status pdx_ivf_build(const float *x, int64_t n, int32_t d, const pdx_ivf_opts *opts,
                         void *stream, pdx_index **out);

/*
 * pdx_search_exact -- exact k-NN of nq queries q[nq][d] over an index built
 * by pdx_build_layout (Sec. 2.1; PDX-BOND, Sec. 5, is exact). Writes
 * out_dist[nq][k] (float32) and out_idx[nq][k] (int64 vector ids). opts may
 * be NULL (PDX-BOND, distance-to-means order). pruner must be NONE, BOND or
 * CS_IP (ADSampling/BSA are approximate and only offered over IVF). IP with
 * BOND requires a unit-norm index (it is searched as L2, the same ranking);
 * CS_IP serves IP indexes of any norms built with cs_first_step.
 * Errors: PDX_ERR_ARG (NULL pointers, nq < 0, k outside [1,1024], bad opts),
 * PDX_ERR_UNSUPPORTED, PDX_ERR_OOM, PDX_ERR_CUDA. nq == 0 is a no-op.
 */
pdx_status pdx_search_exact(const pdx_index *index, const float *q, int64_t nq, int32_t k,
                            const pdx_search_opts *opts, float *out_dist, int64_t *out_idx,
                            void *stream);

/*
 * pdx_search_ivf -- approximate k-NN over an IVF index (Sec. 4, Fig. 4): finds
 * the nprobe buckets whose centroids are nearest to each (transformed) query
 * (ties: lower bucket id), then runs PDXearch over them, nearest bucket first,
 * with the pruner in opts (BOND: exact within the probed buckets). Outputs
 * as pdx_search_exact. Errors: as pdx_search_exact plus PDX_ERR_ARG for
 * nprobe outside [1, nlist] or a pruner that needs a transform the index was
 * not built with.
 */
pdx_status pdx_search_ivf(const pdx_index *index, const float *q, int64_t nq, int32_t k,
                          int32_t nprobe, const pdx_search_opts *opts, float *out_dist,
                          int64_t *out_idx, void *stream);

/*
 * pdx_search_exact_noalloc -- pdx_search_exact for callers that must not
 * allocate device memory during a search. The paper has no counterpart: this
 * exists for hosts that hand the library a fixed memory budget. Examples are a
 * plug-in running inside a process whose device memory is owned by another
 * framework's caching allocator, or a latency-critical serving loop where an
 * allocation (and the implicit synchronisation or pool growth it can cause)
 * must never happen after start-up.
 *
 * The results and errors are those of pdx_search_exact, with these
 * differences:
 *  - q, out_dist and out_idx must be device memory (PDX_ERR_ARG otherwise);
 *    nothing is staged through host memory.
 *  - All scratch (thresholds, per-item candidate lists, START keys, counters)
 *    lives in one file-scope __device__ array of 32 MiB that the library
 *    declares statically. Every GPU that loads the library holds it until the
 *    process exits. A search whose scratch would exceed 32 MiB returns
 *    PDX_ERR_ARG and says how much it needed. Fewer queries per call or a
 *    smaller start_vectors reduce it: about nq*(8*k*parts*groups + 8*start_vectors) bytes.
 *  - The call allocates nothing. It makes no cudaMalloc/cudaFree and uses no
 *    allocating library routine. Every call looks up the array's device
 *    address with cudaGetSymbolAddress, with the calling thread's current
 *    device, so the address stays right after a cudaDeviceReset. The first
 *    call on a device also loads the library's kernels there: make it before
 *    any stream capture. tau_init, if given, must be device memory.
 *  - Every call on a device shares the one array, and each call overwrites it
 *    (the call resets what must start from zero). Calls whose work overlaps
 *    on the GPU (different streams, or host threads without ordering) race
 *    on it and produce wrong results. Serialise them, e.g. on one stream.
 */
pdx_status pdx_search_exact_noalloc(const pdx_index *index, const float *q, int64_t nq, int32_t k,
                                    const pdx_search_opts *opts, float *out_dist, int64_t *out_idx,
                                    void *stream);

/*
 * Batched serving (no counterpart in the paper, which answers one query at a
 * time on one thread): a server answers exact k-NN batches of 1..max_batch
 * queries against any of `count` exact indexes (collections of uneven size and
 * dimensionality). Each (collection, power-of-two batch bucket) pair is
 * prepared on first use. The search is captured as a CUDA graph and replayed
 * afterwards (use_graphs). Its launch shape (resident scan CTAs per SM, first
 * fetch step, i.e. the first prune-check interval, and work-item size in
 * 64-vector blocks: the automatic size, its half and its double) is first
 * chosen by timing candidates on that first batch (autotune). Exact results are identical for every candidate. Tuning
 * results persist in the JSON file tune_cache (optional).
 *
 * The server owns one device workspace sized for its largest plan, plus
 * staging buffers and a private stream. Calls are serialised internally;
 * `stream` orders a call after the caller's prior work, and the caller's
 * stream waits for the results. Host outputs make the call synchronous.
 * Indexes must outlive the server.
 */
typedef struct pdx_server pdx_server;

typedef struct pdx_server_opts {
    uint32_t struct_size;      /* = sizeof(pdx_server_opts)                                */
    int32_t k;                 /* neighbours per query (1..1024)                            */
    int32_t max_batch;         /* largest batch a call may pass (1..65536)                  */
    int32_t use_graphs;        /* capture each (collection, bucket) search in a CUDA graph  */
    int32_t autotune;          /* time candidate launch shapes on first use                 */
    const char *tune_cache;    /* optional JSON file of tuning results (read and written)   */
    pdx_search_opts search;    /* base options; pruner NONE, BOND or CS_IP                 */
} pdx_server_opts;

typedef struct pdx_server_info_t {
    int32_t collections;
    int32_t max_bucket;
    uint64_t workspace_bytes;
    uint64_t graph_launches;   /* batches served by replaying a graph                       */
    uint64_t direct_launches;  /* batches served by direct launches                         */
    uint64_t tunings;          /* (collection, bucket) pairs tuned by timing                */
    int32_t entries_ready;
} pdx_server_info_t;

void pdx_default_server_opts(pdx_server_opts *opts);
/* Errors: PDX_ERR_ARG (NULL/empty, IVF index, k or max_batch out of range, an
 * approximate pruner), PDX_ERR_OOM, PDX_ERR_CUDA. */
pdx_status pdx_server_create(const pdx_index *const *indexes, int32_t count, const pdx_server_opts *opts,
                             pdx_server **out);
/* Exact top-k of nq (1..max_batch) queries q[nq][d] of collection `collection`;
 * outputs as pdx_search_exact. Errors: PDX_ERR_ARG, PDX_ERR_CUDA. */
pdx_status pdx_server_search(pdx_server *server, int32_t collection, const float *q, int64_t nq, float *out_dist,
                             int64_t *out_idx, void *stream);
pdx_status pdx_server_info(const pdx_server *server, pdx_server_info_t *info);
void pdx_server_free(pdx_server *server); /* NULL-safe */

/*
 * Order-proposal network (no counterpart in the paper): u = [q; c] (2d) ->
 * relu(W1 u + b1) (hidden) -> W2 h + b2 (d outputs). A PDX_ORDER_LEARNED search
 * visits dimensions by decreasing (q_j - mu_j)^2 + s_q output_j (s_q =
 * mean_j (q_j - mu_j)^2): the network
 * corrects PDX-BOND's distance-to-means order (mu = collection means); the
 * prune test stays the true partial distance, so results are exact whatever
 * the network proposes.
 * Parameters are one FP32 buffer W1[hidden][2d] | b1[hidden] | W2[d][hidden] |
 * b2[d]; searches use BF16 copies of W1 and W2 with FP32 accumulation.
 * All data pointers below are device memory unless stated; calls synchronise.
 */
pdx_status pdx_mlp_create(int32_t d, int32_t hidden, uint64_t seed, pdx_mlp **out);
void pdx_mlp_free(pdx_mlp *net);
size_t pdx_mlp_param_count(const pdx_mlp *net);
pdx_status pdx_mlp_set_params(pdx_mlp *net, const float *params, size_t count);   /* host or device */
pdx_status pdx_mlp_get_params(const pdx_mlp *net, float *params, size_t count);   /* host or device */
/* y[B][d] = network(u[B][2d]); use_bf16 selects the inference weights. */
pdx_status pdx_mlp_forward(pdx_mlp *net, const float *u, int64_t B, int32_t use_bf16, float *y, void *stream);
/* Gradients of L = sum((y - t)^2) / (B d) into grads (count floats, host or
 * device, parameter layout) and L into *loss (host, optional); FP32 weights. */
pdx_status pdx_mlp_backward(pdx_mlp *net, const float *u, const float *t, int64_t B, float *grads, float *loss,
                            void *stream);
/* Adam (lr, betas 0.9/0.999) over shuffled mini-batches of the n rows (u, t);
 * *loss receives the last epoch's final batch loss. */
pdx_status pdx_mlp_train(pdx_mlp *net, const float *u, const float *t, int64_t n, int32_t epochs, int32_t batch,
                         float lr, uint64_t seed, float *loss, void *stream);
/* Network inputs u[r] = [q_r; c] with c the centroid (row of centroids[nc][d])
 * nearest to q_r in L2 (ties: lower row) -- what a PDX_ORDER_LEARNED search feeds
 * the network. */
pdx_status pdx_mlp_inputs(const float *q, int64_t nq, int32_t d, const float *centroids, int32_t nc, float *u,
                          void *stream);
/* Training targets from the plain method's traces: t[r][j] = mean over the m
 * vectors ids[r][*] (int64, -1 ignored; vectors the plain search pruned for
 * query r) of (q_rj - x_j)^2, minus the heuristic term (q_rj - mu_j)^2 with mu
 * the collection means, divided by s_r = mean_j (q_rj - mu_j)^2. A
 * PDX_ORDER_LEARNED search ranks dimensions by (q_j - mu_j)^2 + s_q network_j,
 * so the network learns the heuristic's error in units of s_q. Exact indexes. */
pdx_status pdx_order_targets(const pdx_index *index, const float *q, int64_t nq, const int64_t *ids, int32_t m,
                             float *targets, void *stream);

/* Release an index and all of its device memory. NULL-safe. */
void pdx_free(pdx_index *index);

/*
 * pdx_merge_topk -- the exchange step of a sharded collection (not in the
 * paper, whose search runs on one machine). Each shard answered the same
 * queries over its own vectors with global ids, best-first as the searches
 * return them; this keeps the k best per query over all shards.
 *   dist, idx  [nshards][nq][k] row-major (padding: idx -1)
 *   metric     order of the lists: L2/L1 ascending, IP descending; ties go
 *              to the lower id and padding comes last
 *   out_*      [nq][k], the same order and padding
 * All four arrays are host pointers (merged on the calling thread; no GPU
 * needed) or all device pointers (one kernel on `stream`, asynchronous).
 * Returns PDX_ERR_ARG for nshards outside [1, 64], k outside [1, 1024], a bad
 * metric, NULL arrays, or a mix of host and device arrays.
 */
pdx_status pdx_merge_topk(const float *dist, const int64_t *idx, int32_t nshards, int64_t nq, int32_t k,
                          pdx_metric metric, float *out_dist, int64_t *out_idx, void *stream);

/* Number of CUDA kernels this process has launched through the library; a
 * server's graph replay counts each kernel node of the graph. */
uint64_t pdx_kernel_launches(void);

/* Message of the last non-OK status on this thread ("" if none). */
const char *pdx_last_error(void);

/* Sizes and flags of an index. */
pdx_status pdx_index_info_get(const pdx_index *index, pdx_index_info *info);

/* Copy one internal array (see pdx_array) to dst (host or device) of `bytes`
 * bytes; PDX_ERR_ARG if bytes differs from the array's size. Synchronous. */
pdx_status pdx_index_copy_out(const pdx_index *index, pdx_array which, void *dst, size_t bytes);

#ifdef __cplusplus
}
#endif

#endif /* PDX_H_ */
