// Internal declarations shared by the CUDA translation units of libpdx.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "pdx.h"

namespace pdx {

// Sec. 3: vectors are grouped in blocks of 64 and stored dimension-major inside
// a block; 64 is the paper's best block size (Table 4) and also two warps'
// worth of 32-bit lanes, so one warp covers a block with one float4 per lane
// per pair of dimensions.
constexpr int kBlock = 64;
constexpr int kMaxSurv = 16;   // PRUNE-phase survivors held in registers (selection <= 25%)
constexpr int kMaxK = 1024;
constexpr int kMaxD = 4096;
constexpr int kMaxSortUnits = 256;  // zone keys a scan warp sorts in-kernel (8 per lane)
constexpr int kPoolCap = 256;       // shared candidate distances per query (8 per lane)
constexpr int kStartProbe = 2;      // start clusters a query's START reads (at least; more for large k)
constexpr int kMaxChecks = 16;      // prune check points of one fetch schedule (doubling: log2(d) + 1)
constexpr int kStartMembers = 64;   // member vectors kept per start cluster

// Device counters, in the order of the first fields of pdx_search_stats
// (slot 7 is bytes_logical, which the host derives and no kernel writes).
enum Counter {
    C_VALUES = 0, C_SCANNED, C_PRUNED, C_PRUNE_BLOCKS, C_CANDIDATES, C_ITEMS, C_START, C_BYTES_HOST,
    C_DENSE_FALLBACK, C_COUNT
};

// Kernels launched through the library (host-side count).
void count_launches(int n);
inline cudaError_t counted(cudaError_t e) {
    if (e == cudaSuccess) count_launches(1);
    return e;
}

}  // namespace pdx

// Opaque handle of the C ABI.
struct pdx_index {
    int64_t n = 0;
    int32_t d = 0;
    pdx_metric metric = PDX_L2;
    pdx_dtype storage = PDX_F32;
    int32_t is_ivf = 0;
    int32_t unit_norm = 0;
    int32_t nparts = 0;
    int64_t nblocks = 0;
    int device = 0;
    pdx_pruner transform = PDX_PRUNE_NONE;  // IVF: ADSAMPLING rotation / BSA projection
    // device arrays
    float *data = nullptr;          // [nblocks][d][64] FP32 (absent for low-precision storage)
    void *data_lp = nullptr;        // [nblocks][d][64] BF16 / FP8-E4M3 blocks
    float *scale = nullptr;         // [d] FP8: per-dimension scale
    float *xnary = nullptr;         // [n][d] FP32 vectors by id (low precision: START, rerank;
                                    // tensor-core dense engine; row finish; canonical refine).
                                    // A rotated or projected IVF index keeps the original
                                    // (untransformed) vectors here.
    float *dsm = nullptr;           // [d][n_pad] fully dimension-major copy (keep_dsm), n_pad = ceil(n/64)*64
    // START clusters (exact indexes): k-means centroids over a sample and, for
    // each, the ids of the sc_m vectors nearest to it among those assigned to it
    int32_t sc_c = 0, sc_m = 0;
    float *sc_cent = nullptr;       // [sc_c][d] row-major
    int32_t *sc_members = nullptr;  // [sc_c][sc_m], -1 = padding
    float *xtc = nullptr;           // [n][d] the rows rounded to TF32 (tensor-core operand)
    float *xnorm = nullptr;         // [n][4] (||x||^2, ||x||, ||x - tf32(x)||, 0) (dense engine)
    int32_t *ids = nullptr;         // [nblocks*64]
    int32_t *slot_of = nullptr;     // [n] storage slot (block*64 + lane) of each vector id
    int32_t *blk_cnt = nullptr;     // [nblocks] valid lanes per block
    int32_t *part_blk = nullptr;    // [nparts+1]
    float *means = nullptr;         // [nparts][d]
    float *vars = nullptr;          // [nparts][d] per-part population variances (IVF: the fused pruner)
    float *cmean = nullptr;         // [d] collection means
    float *centroids = nullptr;     // [nparts][d] (IVF)
    float *centroid_norms = nullptr;// [nparts]
    int32_t *assign = nullptr;      // [n] (IVF)
    float *rot = nullptr;           // [d][d] query transform (row-major, q' = rot * (q - shift))
    float *shift = nullptr;         // [d] (BSA: data mean)
    float *pca_var = nullptr;       // [d] (BSA: variance of each projected dimension)
    float *resid = nullptr;         // BSA: [nblocks][nchk][64] squared residual norms
    int32_t bsa_nchk = 0;           // BSA: number of check points stored
    int32_t bsa_first_step = 4;     // BSA: fetch schedule the residual norms were taken for
    int32_t *chk = nullptr;         // BSA: [bsa_nchk] dimensions visited at each check point
    int32_t cs_first_step = 0;      // CS-IP: fetch schedule of the stored norms (0 = none)
    int32_t cs_nchk = 0;            // CS-IP: check points of that schedule
    int32_t *cs_chk = nullptr;      // CS-IP: [cs_nchk+1] 0, then the dimensions visited at each check
    float *cs_resid = nullptr;      // CS-IP: [nblocks][cs_nchk+1][64] squared norms of the dimensions
                                    //   from cs_chk[t] on (t = 0: the whole vector)
    float *cdata = nullptr;         // IVF centroids in PDX layout [c_nblocks][d][64]
    int32_t *cids = nullptr;        // [c_nblocks*64] bucket id per slot, -1 = padding
    int32_t c_nblocks = 0;
    // host mirrors
    int32_t *h_part_blk = nullptr;  // [nparts+1]
    uint64_t bytes = 0;
};

// Order-proposal network (pdx_mlp.cu).
struct pdx_mlp {
    int d = 0, hidden = 0;
    // FP32 master parameters, one buffer: W1 [H][2D] | b1 [H] | W2 [D][H] | b2 [D]
    float *p = nullptr;
    float *g = nullptr;            // gradients, same layout
    float *m = nullptr, *v = nullptr;  // Adam moments
    uint16_t *w1h = nullptr, *w2h = nullptr;  // BF16 copies of W1, W2 for inference
    bool bf16_stale = true;
    int64_t adam_t = 0;
    size_t count = 0;
    float *w1() const { return p; }
    float *b1() const { return p + (size_t)hidden * 2 * d; }
    float *w2() const { return b1() + hidden; }
    float *b2() const { return w2() + (size_t)d * hidden; }
};

namespace pdx {

void set_error(const char *fmt, ...);
pdx_status cuda_status_ext(cudaError_t e, const char *what);

struct SearchPlan {
    int pruner;
    int metric;      // metric the scan computes (IP on unit vectors is searched as L2)
    int out_mode;    // 0: distance as ranked; 1: IP = -ranked value
};
pdx_status check_search_args(const pdx_index *ix, const float *q, int64_t nq, int32_t k,
                             const pdx_search_opts *opts, float *out_dist, int64_t *out_idx,
                             pdx_search_opts *o, const char *fn);
pdx_status plan_metric(const pdx_index *ix, int pruner, SearchPlan *pl, const char *fn);

// ---- device helpers ----
#ifdef __CUDACC__
// Monotone map float -> uint32 (total order equal to the float order for
// non-NaN values), so (distance, id) pairs sort as one uint64 key.
__device__ __forceinline__ uint32_t f2o(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float o2f(uint32_t o) {
    uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    return __uint_as_float(u);
}
__device__ __forceinline__ uint64_t make_key(float dist, int32_t id) {
    return ((uint64_t)f2o(dist) << 32) | (uint32_t)id;
}
__device__ __forceinline__ float key_dist(uint64_t key) { return o2f((uint32_t)(key >> 32)); }
__device__ __forceinline__ int32_t key_id(uint64_t key) { return (int32_t)(uint32_t)(key & 0xffffffffu); }

enum { MT_L2 = 0, MT_IP = 1, MT_L1 = 2 };
constexpr unsigned kFull = 0xffffffffu;

// Raise a kernel's dynamic shared-memory limit to at least `bytes`, never
// lowering it. Launches of one kernel ask for different sizes (they depend on
// d and k); a limit set lower by a later, smaller launch would make an earlier
// launch with more shared memory (e.g. a kernel node of a captured CUDA graph,
// or its replay under a profiler) invalid.
// One lock for all kernels: two host threads raising the same kernel's limit
// to different sizes must not leave the smaller one in place.
inline std::mutex &smem_limit_lock() {
    static std::mutex m;
    return m;
}
template <typename F>
inline cudaError_t raise_smem_limit(F *func, size_t bytes) {
    std::lock_guard<std::mutex> guard(smem_limit_lock());
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Smallest power of two >= v (v >= 1).
__host__ __device__ inline int pow2_ceil(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// One dimension's contribution to the distance (Sec. 2.1): squared
// difference, product, or absolute difference.
template <int MET>
__device__ __forceinline__ float term(float qv, float x, float acc) {
    if (MET == MT_L2) {
        float t = qv - x;
        return fmaf(t, t, acc);
    } else if (MET == MT_IP) {
        return fmaf(qv, x, acc);
    } else {
        return acc + fabsf(qv - x);
    }
}

// distance used for ranking (smaller is better)
template <int MET>
__device__ __forceinline__ float rank_dist(float acc) { return MET == MT_IP ? -acc : acc; }

// Fixed butterfly: every lane ends with the same sum, in the same order.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
#endif

constexpr uint64_t kEmptyKey = ~0ull;

// ---- launchers (each returns the launch's cudaError_t) ----
cudaError_t launch_to_pdx(const float *x, int32_t d, const int32_t *ids, int64_t nblocks,
                          float *data, cudaStream_t st);
cudaError_t launch_part_means(const float *data, const int32_t *blk_cnt, const int32_t *part_blk,
                              int32_t nparts, int32_t d, float *means, cudaStream_t st);
cudaError_t launch_part_vars(const float *data, const int32_t *blk_cnt, const int32_t *part_blk, int32_t nparts,
                             int32_t d, const float *means, float *vars, cudaStream_t st);
// Visited shares F_q of the expected distance at each check point (fused pruner).
cudaError_t launch_mass(const float *q, int64_t rows, int32_t d, int32_t per_part, const int32_t *row_part,
                        const float *means, const float *vars, const uint16_t *order, const int32_t *chk, int32_t nchk,
                        float *out, cudaStream_t st);
cudaError_t launch_unit_norm_check(const float *x, int64_t n, int32_t d, float tol, int *flag,
                                   cudaStream_t st);
cudaError_t launch_fill_u32(uint32_t *p, uint32_t v, int64_t n, cudaStream_t st);
cudaError_t launch_fill_u64(uint64_t *p, uint64_t v, int64_t n, cudaStream_t st);
cudaError_t launch_add_u64(unsigned long long *p, unsigned long long v, cudaStream_t st);

struct ScanParams {
    const float *data;         // F32 PDX blocks
    const void *data_lp;       // BF16 / FP8 PDX blocks (storage != F32)
    int32_t storage;           // pdx_dtype of the blocks
    const float *scale;        // FP8: per-dimension scale [d]
    const float *xnary;        // low precision: FP32 vectors by id [n][d] for the rerank
    const int32_t *ids;
    const int32_t *blk_cnt;
    const int32_t *part_blk;
    int32_t d;
    const float *q;            // [nq][d] (transformed for ADS/BSA)
    const float *qrows;        // [nq][d] the queries in the space of xnary (untransformed)
    int64_t nq;
    const float *means;        // [nparts][d] (BOND order)
    const int32_t *probes;     // [nq][nslots] part per slot, or null (slot -> part0 + slot/chunks)
    int32_t nslots;            // items per query
    int32_t part0;
    int32_t slot0;             // first slot this launch covers (item w -> slot slot0 + w / nq)
    int32_t chunks_per_part;   // exact search: block groups per partition
    int32_t blocks_per_item;
    int32_t k;
    float *tau;                // [nq]
    uint64_t *cand;            // [nq][nslots][k]
    unsigned long long *counters;
    int *work_counter;
    int64_t nitems;
    int32_t first_step;
    int32_t sel_count;         // PRUNE when survivors <= sel_count
    int32_t zone_dims;
    int32_t order;
    int32_t ctas_per_sm;       // resident CTAs per SM the launch is shaped for
    float gamma;               // relative slack covering FP32 rounding of partial sums
    float eps0;
    float bsa_m;
    const uint16_t *qorder;    // optional precomputed visit orders ([nq] or [nq][nparts] rows of d)
    int32_t qorder_per_part;   // rows indexed by (query, part rank) instead of query
    const float *qaux;         // BSA: [nq][nchk][2] (||q_r||^2, s_d(q)^2) per check point
    const float *resid;        // BSA: [nblocks][nchk][64]
    int32_t nchk;
    // Per-query pool of full distances found by any warp (kPoolCap slots,
    // +inf until written): its k-th smallest is the query's running k-th
    // best over everything scanned so far, as one heap per query would give.
    float *pool;               // [nq][kPoolCap] or null
    int32_t *pool_cnt;         // [nq]
    int32_t tau_fixed;         // thresholds stay at their initial values (no tightening)
    int32_t rows_vec4;         // d % 4 == 0 and xnary, qrows 16-byte aligned: rows read as float4
    uint64_t *fin_log;         // optional: (query << 32) | id of every vector carried through all D
    unsigned long long *fin_count;
    uint64_t fin_cap;
};


cudaError_t launch_scan(int pruner, int metric, const ScanParams &p, int num_sms, cudaStream_t st);
// Visit orders for PDX-BOND (mode 0 distance to means with zones of Z, mode 1
// decreasing query value); per_part > 0: one row per (query, part) with
// means[part], else one row per query with means[0..d).
cudaError_t launch_order(const float *q, int64_t rows, int32_t d, const float *means, int32_t per_part,
                         const int32_t *row_part, int mode, int32_t Z, const float *scores, uint16_t *out,
                         cudaStream_t st);
// learned order: network inputs [q; nearest centroid] and BF16 inference
cudaError_t launch_mlp_inputs(const float *q, int64_t nq, int d, const float *cent, const uint64_t *nearest, float *u,
                              cudaStream_t st);
cudaError_t mlp_scores(pdx_mlp *net, const float *U, int64_t B, float *Z, float *Y, cudaStream_t st);
// learned visit orders [nq][d] in one launch: inputs [q; c], BF16 inference, scores, sort (even hidden size)
cudaError_t mlp_order(pdx_mlp *net, const float *q, int64_t nq, const float *cent, const uint64_t *nearest,
                      const float *mu, uint16_t *order, cudaStream_t st);

// How a search gets its PDX-BOND visit orders (see plan_orders).
struct OrderPlan {
    int mode = -1;        // -1: none precomputed (in-kernel zones or storage order); 0: to means; 1: decreasing;
                          // 2: learned (network scores)
    int per_part = 0;     // >0: rows per query (one per part rank); 0: one row per query
    int64_t rows = 0;
    size_t bytes = 0;
};
OrderPlan plan_orders(const pdx_index *ix, const pdx_search_opts &o, int pruner, int64_t nq, int parts_per_query);

// Exact search split into planning (launch shape, scratch bytes) and running
// (launches only, on caller-provided scratch: no allocation, no sync).
struct ExactPlan {
    int bpi = 1, chunks = 1, nslots = 0;
    bool start = false;
    int start_blk = 0;
    int64_t Lstart = 0;
    OrderPlan op;
    size_t mlp_bytes = 0;      // learned order: centroid keys, nearest, inputs, hidden, scores
    int64_t mlp_Lc = 0;
    int layout = 0;            // pdx_layout of an unpruned scan (0: the PDX scan path)
    bool start_clusters = false;  // START from the query's nearest start clusters
    int64_t sc_ld = 0;         // padded centroid count of the centroid keys
    int32_t sc_probe = 0;      // start clusters read per query: enough members for k
    bool dense = false;        // tensor-core engine (pdx_dense.cu) instead of the scan
    int dense_cap = 0;         // its candidate entries per query
    size_t bytes = 0;
};
pdx_status exact_check(const pdx_index *ix, const float *q, int64_t nq, int32_t k, const pdx_search_opts *opts,
                       float *out_dist, int64_t *out_idx, pdx_search_opts *o, SearchPlan *pl, const char *fn);
pdx_status exact_plan(const pdx_index *ix, int64_t nq, int32_t k, const pdx_search_opts &o, const SearchPlan &pl,
                      int sms, ExactPlan *ep);
// Events recorded on the search stream at the phase boundaries (pdx_search_stats.phase_ns).
struct PhaseEvents {
    cudaEvent_t e[6];
    bool ok;
    PhaseEvents();
    ~PhaseEvents();
    void fill(pdx_search_stats *so) const;
};
pdx_status exact_run(const pdx_index *ix, const float *qd, int64_t nq, int32_t k, const pdx_search_opts &o,
                     const SearchPlan &pl, const ExactPlan &ep, unsigned char *scratch, float *od, int64_t *oi,
                     unsigned long long **counters_out, int sms, cudaStream_t st, const PhaseEvents *ph = nullptr);
void fill_stats(pdx_search_stats *so, const unsigned long long *c, const pdx_index *ix);

// Layout scans (pdx_layouts.cu): linear scans over PDX, N-ary, N-ary + gather
// or DSM storage, merged like the PDX scan's per-item lists.
bool layout_supported(const pdx_index *ix, int layout, int32_t k, const char **why);
size_t layout_scratch_bytes(const pdx_index *ix, int layout, int64_t nq, int32_t k);
pdx_status layout_run(const pdx_index *ix, const float *qd, int64_t nq, int32_t k, int layout, int metric,
                      int out_mode, unsigned char *scratch, float *od, int64_t *oi, int sms, void *ev_start,
                      void *ev_stop, cudaStream_t st);
cudaError_t launch_dsm_transpose(const float *x, int64_t n, int32_t d, int64_t n_pad, float *out, cudaStream_t st);

// Tensor-core dense engine (pdx_dense.cu).
bool dense_supported(const pdx_index *ix, int32_t k, const char **why);
int dense_cap(int64_t n, int32_t k);
size_t dense_scratch_bytes(int64_t nq, int32_t d, int32_t k, int32_t cap, int64_t n, int sms);
pdx_status dense_run(const pdx_index *ix, const float *qd, int64_t nq, int32_t k, int metric, int out_mode,
                     unsigned char *scratch, size_t bytes, int cap, float *od, int64_t *oi, unsigned long long *counters,
                     int sms, void *ev_start, void *ev_stop, cudaStream_t st);
// Tensor-engine operand of x[n][d]: xtc = x rounded to TF32 (to nearest) and
// out[n][4] = (||x||^2, ||x||, ||x - xtc||, 0), sums in FP64, norms rounded up.
cudaError_t launch_dense_operand(const float *x, int64_t n, int32_t d, float *xtc, float *out, cudaStream_t st);
size_t scan_warp_smem(int d, int k, int zone_dims, int order);

// START: exact distances of every query to the first `nvec` stored vectors,
// as (distance, id) keys [nq][nvec_pad].
cudaError_t launch_dense_keys(const float *q, int64_t nq, const float *data, const int32_t *ids,
                              int32_t d, int32_t nblk, int metric, uint64_t *keys, cudaStream_t st);
// START from start clusters: exact distances to the members of each query's
// P nearest clusters (nearest: [nq][P] centroid keys), keys [nq][P*M].
cudaError_t launch_member_keys(const float *q, int64_t nq, int32_t d, const float *rows, const float *data,
                               const int32_t *slot_of, const uint64_t *nearest, int32_t P, const int32_t *members,
                               int32_t M, uint64_t *keys, cudaStream_t st);
// START over row-major FP32 vectors: keys[qi*ld + r] for r < nrows <= ld.
cudaError_t launch_dense_keys_rows(const float *q, int64_t nq, const float *x, int32_t nrows, int32_t d, int64_t ld,
                                   uint64_t *keys, cudaStream_t st);
cudaError_t launch_refine_rows(const uint64_t *topk, int64_t nq, int32_t k, const float *q, int32_t d, const float *x,
                               int metric, uint64_t *out, cudaStream_t st);
cudaError_t launch_fp8_scales(const float *x, int64_t n, int32_t d, unsigned *colmax, float *scale, cudaStream_t st);
cudaError_t launch_quantize(const float *data, int64_t nblocks, int32_t d, int storage, const float *scale, void *out,
                            cudaStream_t st);
// Per-row k smallest keys of a [rows][L] array (sorted ascending) -> out [rows][k].
cudaError_t launch_select_k(const uint64_t *keys, int64_t rows, int64_t L, int32_t k, uint64_t *out,
                            cudaStream_t st);
// The same over keys whose distance is within slack(tau[row], gamma), where
// tau[row] is the row's final threshold (the k-th distance of k real vectors).
// With scratch for at most kSplitSelectRows rows (compact: rows x kSplitSelectCap
// keys, counts: rows ints) a small batch's long rows are first filtered by many
// CTAs at once; null scratch keeps one CTA per row.
constexpr int kSplitSelectRows = 16;
constexpr int kSplitSelectCap = 8192;
cudaError_t launch_select_k_tau(const uint64_t *keys, int64_t rows, int64_t L, int32_t k, const float *tau,
                                float gamma, uint64_t *out, cudaStream_t st, uint64_t *compact, int32_t *counts);
// tau[row] = min(tau[row], init[row]) on the ordered representation.
cudaError_t launch_tau_min(float *tau, const float *init, int64_t rows, cudaStream_t st);
// tau[row] = distance of the k-th key of each row (or +inf).
cudaError_t launch_tau_from_keys(const uint64_t *topk, int64_t rows, int32_t k, float *tau, cudaStream_t st);
// Canonical distances of the selected results: recomputed in the natural
// dimension order with a fixed reduction, in the index's metric, as keys.
cudaError_t launch_refine(const uint64_t *topk, int64_t nq, int32_t k, const float *q, int32_t d,
                          const float *data, const int32_t *slot_of, int metric, uint64_t *out, cudaStream_t st);
// keys -> (float distance, int64 id) outputs. mode 0: dist as is; 1: IP = -dist;
// 2: IP from L2 on unit vectors: (||q||^2 + 1 - L2) / 2.
cudaError_t launch_write_out(const uint64_t *topk, int64_t nq, int32_t k, int mode, const float *q,
                             int32_t d, float *out_dist, int64_t *out_idx, cudaStream_t st);

// IVF
cudaError_t launch_nearest_centroids(const float *x, int64_t n, int32_t d, const float *centroids,
                                     const float *cnorm, int32_t nlist, int32_t *assign, float *best,
                                     cudaStream_t st);
cudaError_t launch_centroid_norms(const float *c, int32_t nlist, int32_t d, float *out, cudaStream_t st);
cudaError_t launch_kmeans_update(const float *x, int64_t n, int32_t d, const int32_t *assign,
                                 int32_t nlist, float *sums, int32_t *counts, float *centroids,
                                 cudaStream_t st);
cudaError_t launch_probe_keys(const float *q, int64_t nq, int32_t d, const float *centroids,
                              int32_t nlist, uint64_t *keys, cudaStream_t st);
cudaError_t launch_keys_to_parts(const uint64_t *topk, int64_t nq, int32_t nprobe, int32_t *probes,
                                 cudaStream_t st);
// y[rows][d] = (x[rows][d] - shift) * M^T   (M row-major d x d), FP32.
cudaError_t launch_transform(const float *x, int64_t rows, int32_t d, const float *M, const float *shift,
                             float *y, cudaStream_t st);
cudaError_t launch_column_stats(const float *x, int64_t n, int32_t d, double *sum, double *gram,
                                cudaStream_t st);
cudaError_t launch_bsa_resid(const float *data, const int32_t *blk_cnt, int64_t nblocks, int32_t d,
                             const int32_t *chk, int32_t nchk, float *resid, cudaStream_t st);
cudaError_t launch_bsa_qaux(const float *q, int64_t nq, int32_t d, const float *var, const int32_t *chk,
                            int32_t nchk, float *qaux, cudaStream_t st);
cudaError_t jacobi_eigen(double *A, double *V, int32_t dd, double *work, int sweeps, cudaStream_t st);
cudaError_t launch_offdiag(const double *A, int32_t dd, double *out, cudaStream_t st);

}  // namespace pdx
