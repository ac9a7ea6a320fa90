// C ABI of libpdx: argument checks, memory management and the host-side
// sequence of kernel launches for each call. See include/pdx.h.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "pdx_internal.cuh"

namespace pdx {

static thread_local std::string g_err;
static std::atomic<unsigned long long> g_launches{0};

// n < 0 takes back launches that a stream capture recorded (modular arithmetic)
void count_launches(int n) { g_launches.fetch_add((unsigned long long)(long long)n, std::memory_order_relaxed); }

void set_error(const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

pdx_status cuda_status_ext(cudaError_t e, const char *what) {
    set_error("%s failed: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PDX_ERR_OOM : PDX_ERR_CUDA;
}

static pdx_status cuda_status(cudaError_t e, const char *what, int line) {
    set_error("%s failed: %s (pdx_api.cu:%d)", what, cudaGetErrorString(e), line);
    return e == cudaErrorMemoryAllocation ? PDX_ERR_OOM : PDX_ERR_CUDA;
}

#define PDX_TRY(call)                                                                                            \
    do {                                                                                                         \
        cudaError_t e_ = (call);                                                                                 \
        if (e_ != cudaSuccess) return ::pdx::cuda_status(e_, #call, __LINE__);                                 \
    } while (0)

static bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static int num_sms() {
    static thread_local int dev_cached = -1, sms = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != dev_cached) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        dev_cached = dev;
    }
    return sms > 0 ? sms : 1;
}

// Stream-ordered scratch: one cudaMallocAsync for all regions of a call,
// released on the same stream when the call returns.
struct Scratch {
    cudaStream_t st;
    void *base = nullptr;
    size_t off = 0, cap = 0;
    explicit Scratch(cudaStream_t s) : st(s) {}
    ~Scratch() {
        if (base) cudaFreeAsync(base, st);
    }
    cudaError_t reserve(size_t bytes) {
        cap = bytes;
        if (bytes == 0) return cudaSuccess;
        return cudaMallocAsync(&base, bytes, st);
    }
    // Carves the next region; returns nullptr (and sets overflow) instead of
    // handing out memory past the reservation.
    bool overflow = false;
    template <class T>
    T *take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        if (off + bytes > cap || (!base && bytes)) {
            overflow = true;
            return nullptr;
        }
        T *p = reinterpret_cast<T *>(static_cast<char *>(base) + off);
        off += bytes;
        return p;
    }
};

#define PDX_CHECK_SCRATCH(scr)                                                                          \
    do {                                                                                                \
        if ((scr).overflow) {                                                                           \
            ::pdx::set_error("internal error: scratch layout exceeds its reservation (pdx_api.cu:%d)", __LINE__); \
            return PDX_ERR_CUDA;                                                                        \
        }                                                                                               \
    } while (0)
static size_t rup(size_t b) { return (b + 255) & ~size_t(255); }

// The scan may read rows (and the matching query rows) as float4 when every
// row starts on a 16-byte boundary.
static int rows_vec4(const pdx_index *ix, const float *qrows) {
    return (ix->d % 4 == 0 && ((uintptr_t)ix->xnary & 15u) == 0 && ((uintptr_t)qrows & 15u) == 0) ? 1 : 0;
}

static void free_index(pdx_index *ix) {
    if (!ix) return;
    void *ptrs[] = {ix->sc_cent, ix->sc_members, ix->data, ix->data_lp, ix->scale, ix->xnary, ix->dsm, ix->xtc, ix->xnorm, ix->ids, ix->slot_of, ix->blk_cnt, ix->part_blk, ix->means, ix->vars, ix->cmean, ix->centroids, ix->centroid_norms,
                    ix->assign, ix->rot, ix->shift, ix->pca_var, ix->resid, ix->chk, ix->cdata, ix->cids,
                    ix->cs_chk, ix->cs_resid};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete[] ix->h_part_blk;
    delete ix;
}

template <class T>
static cudaError_t dalloc(pdx_index *ix, T **p, size_t count) {
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = sizeof(T);
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), bytes);
    if (e == cudaSuccess) ix->bytes += bytes;
    return e;
}

// Lays out `rows` (vector ids, grouped by part) as PDX blocks: part p holds
// rows[part_row[p] .. part_row[p+1]) in that order, in ceil(len/64) blocks.
static pdx_status layout_parts(pdx_index *ix, const float *x_dev, const std::vector<int32_t> &rows,
                               const std::vector<int64_t> &part_row, cudaStream_t st) {
    const int nparts = (int)part_row.size() - 1;
    std::vector<int32_t> part_blk(nparts + 1, 0);
    for (int p = 0; p < nparts; ++p) {
        int64_t len = part_row[p + 1] - part_row[p];
        part_blk[p + 1] = part_blk[p] + (int32_t)((len + kBlock - 1) / kBlock);
    }
    const int64_t nblocks = part_blk[nparts];
    std::vector<int32_t> ids((size_t)nblocks * kBlock, -1), cnt((size_t)(nblocks > 0 ? nblocks : 1), 0);
    std::vector<int32_t> slot_of((size_t)ix->n, -1);
    for (int p = 0; p < nparts; ++p) {
        for (int64_t r = part_row[p]; r < part_row[p + 1]; ++r) {
            int64_t local = r - part_row[p];
            int64_t b = part_blk[p] + local / kBlock;
            ids[(size_t)b * kBlock + local % kBlock] = rows[(size_t)r];
            slot_of[(size_t)rows[(size_t)r]] = (int32_t)(b * kBlock + local % kBlock);
            cnt[(size_t)b] += 1;
        }
    }
    ix->nparts = nparts;
    ix->nblocks = nblocks;
    ix->h_part_blk = new (std::nothrow) int32_t[nparts + 1];
    if (!ix->h_part_blk) {
        set_error("host allocation failed");
        return PDX_ERR_OOM;
    }
    std::memcpy(ix->h_part_blk, part_blk.data(), sizeof(int32_t) * (nparts + 1));
    PDX_TRY(dalloc(ix, &ix->data, (size_t)nblocks * ix->d * kBlock));
    PDX_TRY(dalloc(ix, &ix->ids, (size_t)nblocks * kBlock));
    PDX_TRY(dalloc(ix, &ix->slot_of, (size_t)ix->n));
    PDX_TRY(dalloc(ix, &ix->blk_cnt, (size_t)nblocks));
    PDX_TRY(dalloc(ix, &ix->part_blk, (size_t)nparts + 1));
    PDX_TRY(dalloc(ix, &ix->means, (size_t)nparts * ix->d));
    PDX_TRY(cudaMemcpyAsync(ix->ids, ids.data(), ids.size() * 4, cudaMemcpyHostToDevice, st));
    PDX_TRY(cudaMemcpyAsync(ix->slot_of, slot_of.data(), slot_of.size() * 4, cudaMemcpyHostToDevice, st));
    PDX_TRY(cudaMemcpyAsync(ix->blk_cnt, cnt.data(), (size_t)nblocks * 4, cudaMemcpyHostToDevice, st));
    PDX_TRY(cudaMemcpyAsync(ix->part_blk, part_blk.data(), part_blk.size() * 4, cudaMemcpyHostToDevice, st));
    PDX_TRY(launch_to_pdx(x_dev, ix->d, ix->ids, nblocks, ix->data, st));
    PDX_TRY(launch_part_means(ix->data, ix->blk_cnt, ix->part_blk, nparts, ix->d, ix->means, st));
    // collection means = part means weighted by part sizes
    {
        std::vector<float> hm((size_t)nparts * ix->d);
        PDX_TRY(cudaMemcpyAsync(hm.data(), ix->means, hm.size() * 4, cudaMemcpyDeviceToHost, st));
        PDX_TRY(cudaStreamSynchronize(st));
        std::vector<double> acc((size_t)ix->d, 0.0);
        int64_t tot = 0;
        for (int p = 0; p < nparts; ++p) {
            int64_t len = part_row[p + 1] - part_row[p];
            tot += len;
            for (int j = 0; j < ix->d; ++j) acc[(size_t)j] += (double)hm[(size_t)p * ix->d + j] * (double)len;
        }
        std::vector<float> cm((size_t)ix->d);
        for (int j = 0; j < ix->d; ++j) cm[(size_t)j] = tot ? (float)(acc[(size_t)j] / (double)tot) : 0.f;
        PDX_TRY(dalloc(ix, &ix->cmean, (size_t)ix->d));
        PDX_TRY(cudaMemcpyAsync(ix->cmean, cm.data(), cm.size() * 4, cudaMemcpyHostToDevice, st));
    }
    // host vectors above are pageable: the copies have completed once the stream drains
    PDX_TRY(cudaStreamSynchronize(st));
    return PDX_OK;
}

static bool valid_metric(int m) { return m == PDX_L2 || m == PDX_IP || m == PDX_L1; }

static size_t elem_size(pdx_dtype t) { return t == PDX_F32 ? 4 : (t == PDX_BF16 ? 2 : 1); }

// Low-precision storage: quantise the FP32 PDX blocks (BF16, or FP8-E4M3 with
// per-dimension scales taken from xblk, the vectors as the blocks hold them),
// keep the FP32 vectors by id (xrows, row-major: for a transformed IVF index
// the original vectors) for the START scan and the rerank, and release the
// FP32 blocks.
static pdx_status finish_low_precision(pdx_index *ix, const float *xblk, const float *xrows, cudaStream_t st) {
    const int d = ix->d;
    PDX_TRY(dalloc(ix, &ix->xnary, (size_t)ix->n * d));
    PDX_TRY(cudaMemcpyAsync(ix->xnary, xrows, (size_t)ix->n * d * 4, cudaMemcpyDeviceToDevice, st));
    unsigned *colmax = nullptr;
    if (ix->storage == PDX_FP8_E4M3) {
        PDX_TRY(dalloc(ix, &ix->scale, (size_t)d));
        PDX_TRY(cudaMalloc(&colmax, (size_t)d * 4));
        cudaError_t e = launch_fp8_scales(xblk, ix->n, d, colmax, ix->scale, st);
        if (e != cudaSuccess) {
            cudaFree(colmax);
            return cuda_status(e, "launch_fp8_scales", __LINE__);
        }
    }
    const size_t lp_bytes = (size_t)ix->nblocks * d * kBlock * elem_size(ix->storage);
    cudaError_t e = cudaMalloc(&ix->data_lp, lp_bytes ? lp_bytes : 1);
    if (e == cudaSuccess) {
        ix->bytes += lp_bytes;
        e = launch_quantize(ix->data, ix->nblocks, d, ix->storage, ix->scale, ix->data_lp, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (colmax) cudaFree(colmax);
    if (e != cudaSuccess) return cuda_status(e, "quantize", __LINE__);
    cudaFree(ix->data);
    ix->data = nullptr;
    ix->bytes -= (size_t)ix->nblocks * d * kBlock * 4;
    return PDX_OK;
}

// Row-major FP32 vectors by id (the scan finishes few-survivor PRUNE phases
// from them; low-precision storage keeps them as its rerank source).
static pdx_status keep_rows(pdx_index *ix, const float *xrows, cudaStream_t st) {
    if (ix->xnary) return PDX_OK;
    PDX_TRY(dalloc(ix, &ix->xnary, (size_t)ix->n * ix->d));
    PDX_TRY(cudaMemcpyAsync(ix->xnary, xrows, (size_t)ix->n * ix->d * 4, cudaMemcpyDeviceToDevice, st));
    PDX_TRY(cudaStreamSynchronize(st));
    return PDX_OK;
}

// Check points of the doubling fetch schedule (dimensions visited at each
// prune test): first_step, first_step*3, ... strictly below d.
static std::vector<int32_t> check_points(int d, int first_step) {
    std::vector<int32_t> c;
    int pos = 0, step = std::max(1, first_step);
    while (true) {
        pos = std::min(d, pos + step);
        if (pos >= d) break;
        c.push_back(pos);
        step *= 2;
    }
    return c;
}

// Norms for the Cauchy-Schwarz inner-product bound (PDX_PRUNE_CS_IP): the
// squared norm of every vector (check 0) and of its dimensions from each
// check point of the fetch schedule starting with first_step on.
static pdx_status build_cs_norms(pdx_index *ix, int first_step, cudaStream_t st) {
    std::vector<int32_t> chk = check_points(ix->d, first_step);
    chk.insert(chk.begin(), 0);
    PDX_TRY(dalloc(ix, &ix->cs_chk, chk.size()));
    PDX_TRY(dalloc(ix, &ix->cs_resid, (size_t)ix->nblocks * chk.size() * kBlock));
    PDX_TRY(cudaMemcpyAsync(ix->cs_chk, chk.data(), chk.size() * 4, cudaMemcpyHostToDevice, st));
    PDX_TRY(launch_bsa_resid(ix->data, ix->blk_cnt, ix->nblocks, ix->d, ix->cs_chk, (int32_t)chk.size(), ix->cs_resid,
                             st));
    PDX_TRY(cudaStreamSynchronize(st));
    ix->cs_first_step = first_step;
    ix->cs_nchk = (int32_t)chk.size() - 1;
    return PDX_OK;
}

// START clusters of an exact index: Lloyd's k-means (8 iterations, the IVF
// kernels) over an evenly strided sample of 64 vectors per centroid, every
// vector assigned to its nearest centroid, and per centroid the ids of the
// kStartMembers assigned vectors nearest to it (ties: lower id). A search's
// START takes exact distances to the members of the query's kStartProbe
// nearest centroids: real vectors near the query, so the initial threshold is
// already close to the final k-th distance.
static pdx_status build_start_clusters(pdx_index *ix, const float *xd, int32_t C, cudaStream_t st) {
    const int64_t n = ix->n;
    const int d = ix->d;
    const int64_t m = std::min<int64_t>(n, (int64_t)C * 64);
    const int64_t stride = n / m;
    Scratch scr(st);
    PDX_TRY(scr.reserve(rup((size_t)m * d * 4) + rup((size_t)C * d * 4) + rup((size_t)C * 4) + rup((size_t)n * 4) +
                        rup((size_t)n * 4)));
    float *sample = scr.take<float>((size_t)m * d);
    float *sums = scr.take<float>((size_t)C * d);
    int32_t *counts = scr.take<int32_t>((size_t)C);
    int32_t *assign = scr.take<int32_t>((size_t)n);
    float *best = scr.take<float>((size_t)n);
    PDX_CHECK_SCRATCH(scr);
    PDX_TRY(cudaMemcpy2DAsync(sample, (size_t)d * 4, xd, (size_t)stride * d * 4, (size_t)d * 4, (size_t)m,
                              cudaMemcpyDeviceToDevice, st));
    PDX_TRY(dalloc(ix, &ix->sc_cent, (size_t)C * d));
    PDX_TRY(cudaMemcpy2DAsync(ix->sc_cent, (size_t)d * 4, sample, (size_t)(m / C) * d * 4, (size_t)d * 4, (size_t)C,
                              cudaMemcpyDeviceToDevice, st));
    for (int it = 0; it < 8; ++it) {
        PDX_TRY(launch_nearest_centroids(sample, m, d, ix->sc_cent, nullptr, C, assign, nullptr, st));
        PDX_TRY(launch_kmeans_update(sample, m, d, assign, C, sums, counts, ix->sc_cent, st));
    }
    PDX_TRY(launch_nearest_centroids(xd, n, d, ix->sc_cent, nullptr, C, assign, best, st));
    std::vector<int32_t> ha((size_t)n);
    std::vector<float> hb((size_t)n);
    PDX_TRY(cudaMemcpyAsync(ha.data(), assign, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
    PDX_TRY(cudaMemcpyAsync(hb.data(), best, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
    PDX_TRY(cudaStreamSynchronize(st));
    std::vector<std::vector<std::pair<float, int32_t>>> per((size_t)C);
    for (int64_t i = 0; i < n; ++i) per[(size_t)ha[(size_t)i]].push_back({hb[(size_t)i], (int32_t)i});
    const int M = kStartMembers;
    std::vector<int32_t> mem((size_t)C * M, -1);
    for (int c = 0; c < C; ++c) {
        auto &v = per[(size_t)c];
        const size_t take = std::min<size_t>(v.size(), (size_t)M);
        std::partial_sort(v.begin(), v.begin() + take, v.end());
        for (size_t i = 0; i < take; ++i) mem[(size_t)c * M + i] = v[i].second;
    }
    PDX_TRY(dalloc(ix, &ix->sc_members, mem.size()));
    PDX_TRY(cudaMemcpyAsync(ix->sc_members, mem.data(), mem.size() * 4, cudaMemcpyHostToDevice, st));
    PDX_TRY(cudaStreamSynchronize(st));
    ix->sc_c = C;
    ix->sc_m = M;
    return PDX_OK;
}

// Tensor-core dense engine: the exact row-major FP32 vectors (rerank; already
// there for low-precision storage), their TF32-rounded copy (the GEMM
// operand) and per-row norms.
static pdx_status keep_dense_rows(pdx_index *ix, const float *xrows, cudaStream_t st) {
    const int d = ix->d;
    if (!ix->xnary) {
        PDX_TRY(dalloc(ix, &ix->xnary, (size_t)ix->n * d));
        PDX_TRY(cudaMemcpyAsync(ix->xnary, xrows, (size_t)ix->n * d * 4, cudaMemcpyDeviceToDevice, st));
    }
    PDX_TRY(dalloc(ix, &ix->xtc, (size_t)ix->n * d));
    PDX_TRY(dalloc(ix, &ix->xnorm, (size_t)ix->n * 4));
    PDX_TRY(launch_dense_operand(ix->xnary, ix->n, d, ix->xtc, ix->xnorm, st));
    PDX_TRY(cudaStreamSynchronize(st));
    return PDX_OK;
}

}  // namespace pdx

using namespace pdx;

extern "C" {

void pdx_default_build_opts(pdx_build_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->struct_size = sizeof *o;
    o->metric = PDX_L2;
    o->storage = PDX_F32;
    o->partition_size = 10000;
    o->keep_rows = 1;
}

void pdx_default_ivf_opts(pdx_ivf_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->struct_size = sizeof *o;
    pdx_default_build_opts(&o->base);
    o->nlist = 1024;
    o->kmeans_iters = 10;
    o->kmeans_sample = 0;
    o->seed = 2503;
    o->transform = PDX_PRUNE_NONE;
}

void pdx_default_search_opts(pdx_search_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->struct_size = sizeof *o;
    o->pruner = PDX_PRUNE_BOND;
    o->order = PDX_ORDER_DIST_TO_MEANS;
    o->zone_dims = 0;
    o->selection_threshold = 0.20f;
    o->eps0 = 2.1f;
    o->bsa_m = 1.0f;
    o->first_step = 4;
    o->means_scope = PDX_MEANS_AUTO;
    o->ctas_per_sm = 0;
    o->start_vectors = 1024;
    o->blocks_per_item = 0;
    o->stats_out = nullptr;
}

const char *pdx_last_error(void) { return g_err.c_str(); }

uint64_t pdx_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

void pdx_free(pdx_index *index) { free_index(index); }

pdx_status pdx_index_info_get(const pdx_index *ix, pdx_index_info *info) {
    if (!ix || !info) {
        set_error("pdx_index_info_get: NULL argument");
        return PDX_ERR_ARG;
    }
    info->n = ix->n;
    info->d = ix->d;
    info->nparts = ix->nparts;
    info->nblocks = ix->nblocks;
    info->metric = ix->metric;
    info->storage = ix->storage;
    info->is_ivf = ix->is_ivf;
    info->unit_norm = ix->unit_norm;
    info->device_bytes = ix->bytes;
    return PDX_OK;
}

pdx_status pdx_index_copy_out(const pdx_index *ix, pdx_array which, void *dst, size_t bytes) {
    if (!ix || !dst) {
        set_error("pdx_index_copy_out: NULL argument");
        return PDX_ERR_ARG;
    }
    const void *src = nullptr;
    size_t need = 0;
    switch (which) {
    case PDX_ARRAY_BLOCKS: src = ix->data; need = (size_t)ix->nblocks * ix->d * kBlock * 4; break;
    case PDX_ARRAY_BLOCKS_LP:
        src = ix->data_lp;
        need = (size_t)ix->nblocks * ix->d * kBlock * elem_size(ix->storage);
        break;
    case PDX_ARRAY_SCALES: src = ix->scale; need = (size_t)ix->d * 4; break;
    case PDX_ARRAY_IDS: src = ix->ids; need = (size_t)ix->nblocks * kBlock * 4; break;
    case PDX_ARRAY_PART_BLOCKS: src = ix->part_blk; need = ((size_t)ix->nparts + 1) * 4; break;
    case PDX_ARRAY_MEANS: src = ix->means; need = (size_t)ix->nparts * ix->d * 4; break;
    case PDX_ARRAY_CENTROIDS: src = ix->centroids; need = (size_t)ix->nparts * ix->d * 4; break;
    case PDX_ARRAY_ASSIGN: src = ix->assign; need = (size_t)ix->n * 4; break;
    case PDX_ARRAY_ROTATION: src = ix->rot; need = (size_t)ix->d * ix->d * 4; break;
    case PDX_ARRAY_VARIANCES: src = ix->pca_var; need = (size_t)ix->d * 4; break;
    case PDX_ARRAY_ROWS: src = ix->xnary; need = (size_t)ix->n * ix->d * 4; break;
    default: set_error("pdx_index_copy_out: unknown array %d", (int)which); return PDX_ERR_ARG;
    }
    if (!src) {
        set_error("pdx_index_copy_out: array %d not present in this index", (int)which);
        return PDX_ERR_ARG;
    }
    if (bytes != need) {
        set_error("pdx_index_copy_out: array %d has %zu bytes, got %zu", (int)which, need, bytes);
        return PDX_ERR_ARG;
    }
    PDX_TRY(cudaMemcpy(dst, src, need, cudaMemcpyDefault));
    return PDX_OK;
}

pdx_status pdx_build_layout(const float *x, int64_t n, int32_t d, const pdx_build_opts *opts, void *stream,
                            pdx_index **out) {
    if (out) *out = nullptr;
    if (!x || !out) {
        set_error("pdx_build_layout: NULL x or out");
        return PDX_ERR_ARG;
    }
    if (n < 1 || n >= (int64_t)1 << 31 || d < 1 || d > kMaxD) {
        set_error("pdx_build_layout: n=%lld d=%d out of range", (long long)n, d);
        return PDX_ERR_ARG;
    }
    pdx_build_opts o;
    pdx_default_build_opts(&o);
    if (opts) {
        if (opts->struct_size < sizeof(pdx_build_opts)) {
            set_error("pdx_build_layout: opts->struct_size %u < %zu", opts->struct_size, sizeof(pdx_build_opts));
            return PDX_ERR_ARG;
        }
        o = *opts;
    }
    if (!valid_metric(o.metric) || (o.storage != PDX_F32 && o.storage != PDX_BF16 && o.storage != PDX_FP8_E4M3)) {
        set_error("pdx_build_layout: bad metric %d or storage %d", (int)o.metric, (int)o.storage);
        return PDX_ERR_ARG;
    }
    if (o.storage != PDX_F32 && o.metric == PDX_L1) {
        set_error("pdx_build_layout: low-precision storage supports L2 (and unit-norm IP) only");
        return PDX_ERR_UNSUPPORTED;
    }
    if (o.partition_size == 0) o.partition_size = 10000;
    if (o.start_clusters < -1) {
        set_error("pdx_build_layout: start_clusters=%d (0 automatic, -1 none, or a count)", o.start_clusters);
        return PDX_ERR_ARG;
    }
    if (o.cs_first_step < 0 || o.cs_first_step > d) {
        set_error("pdx_build_layout: cs_first_step=%d outside [0, d=%d]", o.cs_first_step, d);
        return PDX_ERR_ARG;
    }
    if (o.cs_first_step > 0 && (o.metric != PDX_IP || o.storage != PDX_F32)) {
        set_error("pdx_build_layout: cs_first_step needs metric PDX_IP and FP32 storage");
        return PDX_ERR_UNSUPPORTED;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    pdx_index *ix = new (std::nothrow) pdx_index();
    if (!ix) {
        set_error("host allocation failed");
        return PDX_ERR_OOM;
    }
    ix->n = n;
    ix->d = d;
    ix->metric = o.metric;
    ix->storage = o.storage;
    cudaGetDevice(&ix->device);
    pdx_status s = PDX_OK;
    {
        Scratch scr(st);
        const float *xd = x;
        if (!is_device_ptr(x)) {
            cudaError_t e = scr.reserve(rup((size_t)n * d * 4));
            if (e != cudaSuccess) { free_index(ix); return cuda_status(e, "cudaMallocAsync", __LINE__); }
            float *tmp = scr.take<float>((size_t)n * d);
            if (!tmp) { free_index(ix); set_error("internal error: scratch layout"); return PDX_ERR_CUDA; }
            e = cudaMemcpyAsync(tmp, x, (size_t)n * d * 4, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) { free_index(ix); return cuda_status(e, "cudaMemcpyAsync", __LINE__); }
            xd = tmp;
        }
        // Sec. 6.6: equal horizontal partitions of at most partition_size vectors
        const int64_t nparts = (n + o.partition_size - 1) / o.partition_size;
        const int64_t size = (n + nparts - 1) / nparts;
        std::vector<int64_t> part_row((size_t)nparts + 1);
        for (int64_t p = 0; p <= nparts; ++p) part_row[(size_t)p] = std::min<int64_t>(n, p * size);
        std::vector<int32_t> rows((size_t)n);
        for (int64_t i = 0; i < n; ++i) rows[(size_t)i] = (int32_t)i;
        s = layout_parts(ix, xd, rows, part_row, st);
        if (s == PDX_OK && o.metric == PDX_IP) {
            int *flag = nullptr;
            cudaError_t e = cudaMalloc(&flag, sizeof(int));
            int one = 1;
            if (e == cudaSuccess) e = cudaMemcpy(flag, &one, sizeof one, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = launch_unit_norm_check(xd, n, d, 1e-5f, flag, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&one, flag, sizeof one, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (flag) cudaFree(flag);
            if (e != cudaSuccess) s = cuda_status(e, "unit norm check", __LINE__);
            ix->unit_norm = one;
        }
        if (s == PDX_OK) {
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) s = cuda_status(e, "cudaStreamSynchronize", __LINE__);
        }
        if (s == PDX_OK) {  // START clusters (0: automatic, one per 4096 vectors from 64k vectors on)
            int32_t C = o.start_clusters;
            if (C == 0) C = n >= 65536 ? (int32_t)std::min<int64_t>(1024, n / 4096) : 0;
            if (C > 0) s = build_start_clusters(ix, xd, (int32_t)std::min<int64_t>(C, n), st);
        }
        if (s == PDX_OK && o.cs_first_step > 0) s = build_cs_norms(ix, o.cs_first_step, st);
        if (s == PDX_OK && o.keep_dsm) {  // the fully dimension-major copy (DSM layout scan)
            const int64_t n_pad = (n + kBlock - 1) / kBlock * kBlock;
            cudaError_t e = dalloc(ix, &ix->dsm, (size_t)n_pad * d);
            if (e == cudaSuccess) e = launch_dsm_transpose(xd, n, d, n_pad, ix->dsm, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) s = cuda_status(e, "DSM copy", __LINE__);
        }
        if (s == PDX_OK && o.storage != PDX_F32) s = finish_low_precision(ix, xd, xd, st);
        if (s == PDX_OK && o.storage == PDX_F32 && o.keep_rows) s = keep_rows(ix, xd, st);
        if (s == PDX_OK && o.dense_rows) s = keep_dense_rows(ix, xd, st);
    }
    if (s != PDX_OK) {
        free_index(ix);
        return s;
    }
    *out = ix;
    return PDX_OK;
}

}  // extern "C"

namespace pdx {

pdx_status check_search_args(const pdx_index *ix, const float *q, int64_t nq, int32_t k,
                                    const pdx_search_opts *opts, float *out_dist, int64_t *out_idx,
                                    pdx_search_opts *o, const char *fn) {
    if (!ix || (nq > 0 && (!q || !out_dist || !out_idx))) {
        set_error("%s: NULL argument", fn);
        return PDX_ERR_ARG;
    }
    if (nq < 0 || nq >= (int64_t)1 << 31 || k < 1 || k > kMaxK) {
        set_error("%s: nq=%lld k=%d out of range", fn, (long long)nq, k);
        return PDX_ERR_ARG;
    }
    pdx_default_search_opts(o);
    if (opts) {
        if (opts->struct_size < sizeof(pdx_search_opts)) {
            set_error("%s: opts->struct_size %u < %zu", fn, opts->struct_size, sizeof(pdx_search_opts));
            return PDX_ERR_ARG;
        }
        *o = *opts;
    }
    if (o->pruner < PDX_PRUNE_NONE || o->pruner > PDX_PRUNE_CS_IP || o->order < PDX_ORDER_DIST_TO_MEANS ||
        o->order > PDX_ORDER_LEARNED) {
        set_error("%s: bad pruner %d or order %d", fn, (int)o->pruner, (int)o->order);
        return PDX_ERR_ARG;
    }
    if (o->means_scope != PDX_MEANS_BLOCK && o->means_scope != PDX_MEANS_COLLECTION &&
        o->means_scope != PDX_MEANS_AUTO) {
        set_error("%s: bad means_scope %d", fn, (int)o->means_scope);
        return PDX_ERR_ARG;
    }
    if (!(o->selection_threshold >= 0.f && o->selection_threshold <= 0.25f) || o->first_step < 1 ||
        !(o->eps0 >= 0.f) || !(o->bsa_m >= 0.f) || o->ctas_per_sm > 32) {
        set_error("%s: selection_threshold must be in [0, 0.25], first_step >= 1, eps0/bsa_m >= 0, "
                  "ctas_per_sm <= 32", fn);
        return PDX_ERR_ARG;
    }
    if (o->order == PDX_ORDER_LEARNED &&
        (!o->mlp || !o->mlp_centroids || o->mlp_ncentroids < 1 || pdx_mlp_param_count(o->mlp) == 0 || ix->is_ivf)) {
        set_error("%s: the learned order needs an exact index, a network and its centroids", fn);
        return PDX_ERR_ARG;
    }
    if (o->engine < PDX_ENGINE_AUTO || o->engine > PDX_ENGINE_TENSOR) {
        set_error("%s: bad engine %d", fn, (int)o->engine);
        return PDX_ERR_ARG;
    }
    if (o->layout < PDX_LAYOUT_PDX || o->layout > PDX_LAYOUT_DSM) {
        set_error("%s: bad layout %d", fn, (int)o->layout);
        return PDX_ERR_ARG;
    }
    if (o->tau_fixed && !o->tau_init) {
        set_error("%s: tau_fixed needs tau_init", fn);
        return PDX_ERR_ARG;
    }
    if (o->finished_log &&
        (!o->finished_count || !is_device_ptr(o->finished_log) || !is_device_ptr(o->finished_count))) {
        set_error("%s: finished_log and finished_count must both be device pointers", fn);
        return PDX_ERR_ARG;
    }
    if (o->finished_log && (ix->storage != PDX_F32 || (o->pruner != PDX_PRUNE_BOND && o->pruner != PDX_PRUNE_CS_IP))) {
        set_error("%s: finished_log is kept by FP32 PDX-BOND and CS_IP scans", fn);
        return PDX_ERR_UNSUPPORTED;
    }
    if (o->order == PDX_ORDER_LEARNED && o->mlp->d != ix->d) {
        set_error("%s: the network was built for d=%d, the index has d=%d", fn, o->mlp->d, ix->d);
        return PDX_ERR_ARG;
    }
    // resolve the automatic choices
    if (o->means_scope == PDX_MEANS_AUTO) o->means_scope = ix->is_ivf ? PDX_MEANS_BLOCK : PDX_MEANS_COLLECTION;
    if (o->zone_dims == 0) o->zone_dims = (o->means_scope == PDX_MEANS_COLLECTION) ? 1 : 8;
    // ctas_per_sm 0: the scan's own default (4 for FP32 blocks, 3 for BF16/FP8)
    return PDX_OK;
}

pdx_status plan_metric(const pdx_index *ix, int pruner, SearchPlan *pl, const char *fn) {
    pl->pruner = pruner;
    pl->metric = ix->metric;
    pl->out_mode = 0;
    if (pruner == PDX_PRUNE_CS_IP && ix->metric != PDX_IP) {
        set_error("%s: the Cauchy-Schwarz bound (PDX_PRUNE_CS_IP) is for inner-product indexes", fn);
        return PDX_ERR_UNSUPPORTED;
    }
    if (ix->metric == PDX_IP) {
        if (pruner == PDX_PRUNE_NONE || pruner == PDX_PRUNE_CS_IP) {
            pl->out_mode = 1;   // ranks by -q.x, which holds for any norms under this bound
        } else if (ix->unit_norm) {
            // unit-norm vectors: ||q - x||^2 = ||q||^2 + 1 - 2 q.x ranks like -q.x
            pl->metric = PDX_L2;
            pl->out_mode = 1;   // the refine step recomputes the inner product itself
        } else {
            set_error("%s: pruned inner-product search needs a unit-norm index", fn);
            return PDX_ERR_UNSUPPORTED;
        }
    }
    if (ix->storage != PDX_F32) {
        // low-precision scans bound and rerank L2 distances
        if (ix->metric == PDX_IP && ix->unit_norm) {
            pl->metric = PDX_L2;
            pl->out_mode = 1;
        } else if (ix->metric != PDX_L2) {
            set_error("%s: low-precision storage supports L2 and unit-norm IP only", fn);
            return PDX_ERR_UNSUPPORTED;
        }
    }
    if (pl->metric == PDX_L1 && pruner > PDX_PRUNE_BOND) {
        set_error("%s: ADSampling/BSA are defined for L2 only", fn);
        return PDX_ERR_UNSUPPORTED;
    }
    return PDX_OK;
}

// PDX-BOND visit orders: coarse zones against block means are sorted inside
// the scan kernel; orders that do not depend on the block (collection means,
// decreasing query value) are computed once per query; fine orders against
// block means (more than kMaxSortUnits zones) once per (query, part rank).
OrderPlan plan_orders(const pdx_index *ix, const pdx_search_opts &o, int pruner, int64_t nq, int parts_per_query) {
    OrderPlan pl;
    const int d = ix->d;
    if (pruner == PDX_PRUNE_ADS_BOND) {
        // the fused pruner: distance-to-means zones against each probed
        // bucket's means, one row per (query, bucket), for the scan and F_q
        pl.mode = 0;
        pl.per_part = parts_per_query;
        pl.rows = nq * pl.per_part;
        pl.bytes = (size_t)pl.rows * d * 2;
        return pl;
    }
    if (pruner != PDX_PRUNE_BOND || o.order == PDX_ORDER_SEQUENTIAL) return pl;
    if (o.order == PDX_ORDER_LEARNED) {
        pl.mode = 2;
    } else if (o.order == PDX_ORDER_DECREASING) {
        pl.mode = 1;
    } else if (o.means_scope == PDX_MEANS_COLLECTION) {
        pl.mode = 0;
    } else {
        int z = o.zone_dims < 1 ? 1 : (int)o.zone_dims;
        if ((d + z - 1) / z <= kMaxSortUnits) return pl;
        pl.mode = 0;
        pl.per_part = parts_per_query;
    }
    pl.rows = pl.per_part ? nq * pl.per_part : nq;
    pl.bytes = (size_t)pl.rows * d * 2;
    return pl;
}

}  // namespace pdx

namespace pdx {

// Launch shape and scratch layout of an exact search (no allocation).
pdx_status exact_plan(const pdx_index *ix, int64_t nq, int32_t k, const pdx_search_opts &o, const SearchPlan &pl,
                      int sms, ExactPlan *ep) {
    // work items: (query, partition, block group); split partitions when
    // there are too few (query, partition) pairs to fill the GPU
    int max_blk = 0;
    for (int p = 0; p < ix->nparts; ++p) max_blk = std::max(max_blk, ix->h_part_blk[p + 1] - ix->h_part_blk[p]);
    int bpi = (int)o.blocks_per_item;
    if (bpi <= 0) {
        const int64_t target = (int64_t)sms * 64 * 3;
        int64_t pairs = std::max<int64_t>(1, nq * (int64_t)ix->nparts);
        int64_t want = std::max<int64_t>(1, (target + pairs - 1) / pairs);
        // each item leaves a k-entry list per query for the merge: keep the
        // lists of one query within 256k keys
        want = std::min<int64_t>(want, std::max<int64_t>(1, ((int64_t)1 << 18) / ((int64_t)ix->nparts * k)));
        int chunks = (int)std::min<int64_t>(max_blk, want);
        bpi = (max_blk + chunks - 1) / chunks;
    }
    if (bpi < 1) bpi = 1;
    ep->bpi = bpi;
    ep->chunks = (max_blk + bpi - 1) / bpi;
    // linear scan over another storage layout (the layout comparison)
    if (o.layout != PDX_LAYOUT_PDX) {
        const char *why = nullptr;
        if (pl.pruner != PDX_PRUNE_NONE || o.engine == PDX_ENGINE_TENSOR) {
            set_error("layout %d: layout scans are unpruned scans (pruner NONE, engine SCAN or AUTO)", (int)o.layout);
            return PDX_ERR_UNSUPPORTED;
        }
        if (!layout_supported(ix, o.layout, k, &why)) {
            set_error("layout %d: %s", (int)o.layout, why);
            return PDX_ERR_UNSUPPORTED;
        }
        ep->layout = (int)o.layout;
        ep->bytes = layout_scratch_bytes(ix, o.layout, nq, k) + rup(C_COUNT * 8);
        return PDX_OK;
    }
    // unpruned search: the tensor-core engine when the index supports it
    const char *why = nullptr;
    const bool can_dense = pl.pruner == PDX_PRUNE_NONE && dense_supported(ix, k, &why);
    if (o.engine == PDX_ENGINE_TENSOR && !can_dense) {
        set_error("tensor-core engine: %s",
                  pl.pruner != PDX_PRUNE_NONE ? "it runs unpruned searches only (pruner PDX_PRUNE_NONE)" : why);
        return PDX_ERR_UNSUPPORTED;
    }
    // AUTO: the GEMM's fixed cost (two passes, select, finish) pays off once
    // the product is large; small searches (e.g. 100 x 10k x 128) run faster
    // on the scan
    const bool big = (double)nq * (double)ix->n * (double)ix->d >= 4294967296.0;
    ep->dense = can_dense && (o.engine == PDX_ENGINE_TENSOR || (o.engine == PDX_ENGINE_AUTO && big));
    if (ep->dense) {
        ep->dense_cap = dense_cap(ix->n, k);
        ep->nslots = 0;
        ep->bytes = dense_scratch_bytes(nq, ix->d, k, ep->dense_cap, ix->n, sms) + rup(C_COUNT * 8);
        return PDX_OK;
    }
    ep->nslots = ix->nparts * ep->chunks;
    ep->start = (pl.pruner != PDX_PRUNE_NONE) && !o.tau_fixed;
    ep->start_blk = 0;
    // START from the query's nearest start clusters when the index has them
    // (L2 ranking), else from the first start_vectors stored vectors
    ep->start_clusters = ep->start && ix->sc_c > 0 && pl.metric == PDX_L2;
    ep->sc_ld = ep->start_clusters ? ((int64_t)ix->sc_c + kBlock - 1) / kBlock * kBlock : 0;
    // kStartProbe clusters, or enough for twice k members (k = 100: 4), at
    // most 16 and at most all of them: the initial threshold is the k-th of
    // the members' distances, which is loose when k is close to their count
    ep->sc_probe = 0;
    if (ep->start_clusters) {
        const int want = (2 * k + ix->sc_m - 1) / ix->sc_m;
        ep->sc_probe = std::min(std::min(16, ix->sc_c), std::max(kStartProbe, want));
    }
    if (ep->start && !ep->start_clusters) {
        int64_t sv = std::max<int64_t>(o.start_vectors, k);
        ep->start_blk = (int)std::min<int64_t>(ix->nblocks, (sv + kBlock - 1) / kBlock);
    }
    ep->Lstart = (int64_t)ep->start_blk * kBlock;
    ep->op = plan_orders(ix, o, pl.pruner, nq, ix->nparts);

    size_t b = rup((size_t)nq * 4)                              // tau
               + rup((size_t)nq * ep->nslots * k * 8)           // per-item lists
               + 3 * rup((size_t)nq * k * 8)                    // merged, refined, final top-k
               + rup(C_COUNT * 8) + rup(8)                      // counters, work counter
               + rup(ep->op.bytes)                              // visit orders
               + rup((size_t)nq * kPoolCap * 4) + rup((size_t)nq * 4);  // shared candidate pools
    if (ep->start) b += rup((size_t)nq * ep->Lstart * 8) + rup((size_t)nq * k * 8);
    if (ep->start_clusters)
        b += rup((size_t)nq * ep->sc_ld * 8) + rup((size_t)nq * ep->sc_probe * 8) +
             rup((size_t)nq * ep->sc_probe * ix->sc_m * 8);
    if (o.tau_init) b += rup((size_t)nq * 4);
    if (nq <= kSplitSelectRows)  // the final selection's compact buffer and counters
        b += rup((size_t)nq * kSplitSelectCap * 8) + rup((size_t)nq * 4);
    if (pl.pruner == PDX_PRUNE_CS_IP) {
        if ((int)o.first_step != ix->cs_first_step) {
            set_error("PDX_PRUNE_CS_IP: first_step %u differs from the index's stored schedule (%d)", o.first_step,
                      ix->cs_first_step);
            return PDX_ERR_ARG;
        }
        b += rup((size_t)nq * (ix->cs_nchk + 1) * 2 * 4);  // the query's norms at the check points
    }
    ep->mlp_bytes = 0;
    if (ep->op.mode == 2) {
        ep->mlp_Lc = ((int64_t)o.mlp_ncentroids + kBlock - 1) / kBlock * kBlock;
        const int hidden = o.mlp->hidden;
        ep->mlp_bytes = rup((size_t)nq * ep->mlp_Lc * 8) + rup((size_t)nq * 8) + rup((size_t)nq * 2 * ix->d * 4) +
                        rup((size_t)nq * hidden * 4) + rup((size_t)nq * ix->d * 4);
    }
    b += ep->mlp_bytes;
    ep->bytes = b;
    return PDX_OK;
}

// All launches of an exact search on `st`, with scratch carved from
// `scratch` (ep.bytes, 256-byte aligned). Allocates nothing and does not
// synchronise, so it can be captured in a CUDA graph (without scan events).
pdx_status exact_run(const pdx_index *ix, const float *qd, int64_t nq, int32_t k, const pdx_search_opts &o,
                     const SearchPlan &pl, const ExactPlan &ep, unsigned char *scratch, float *od, int64_t *oi,
                     unsigned long long **counters_out, int sms, cudaStream_t st, const PhaseEvents *ph) {
    const int d = ix->d;
    auto mark = [&](int i) -> cudaError_t { return ph ? cudaEventRecord(ph->e[i], st) : cudaSuccess; };
    PDX_TRY(mark(0));
    if (ep.layout != PDX_LAYOUT_PDX) {
        const size_t lb = layout_scratch_bytes(ix, ep.layout, nq, k);
        unsigned long long *counters = reinterpret_cast<unsigned long long *>(scratch + lb);
        PDX_TRY(cudaMemsetAsync(counters, 0, C_COUNT * 8, st));
        unsigned long long *kc = o.stats_device ? reinterpret_cast<unsigned long long *>(o.stats_device) : counters;
        if (counters_out) *counters_out = kc;
        // every value of every vector is visited
        PDX_TRY(launch_add_u64(kc + C_VALUES, (unsigned long long)nq * ix->n * d, st));
        PDX_TRY(launch_add_u64(kc + C_SCANNED, (unsigned long long)nq * ix->n, st));
        for (int i = 1; i <= 3; ++i) PDX_TRY(mark(i));
        pdx_status ls = layout_run(ix, qd, nq, k, ep.layout, pl.metric, pl.out_mode, scratch, od, oi, sms,
                                   o.scan_event_start, o.scan_event_stop, st);
        if (ls != PDX_OK) return ls;
        PDX_TRY(mark(4));
        PDX_TRY(mark(5));
        return PDX_OK;
    }
    if (ep.dense) {
        const size_t db = dense_scratch_bytes(nq, d, k, ep.dense_cap, ix->n, sms);
        unsigned long long *counters = reinterpret_cast<unsigned long long *>(scratch + db);
        PDX_TRY(cudaMemsetAsync(counters, 0, C_COUNT * 8, st));
        unsigned long long *kc = o.stats_device ? reinterpret_cast<unsigned long long *>(o.stats_device) : counters;
        if (counters_out) *counters_out = kc;
        const bool ip = ix->metric == PDX_IP;
        for (int i = 1; i <= 3; ++i) PDX_TRY(mark(i));
        pdx_status ds = dense_run(ix, qd, nq, k, ip ? MT_IP : MT_L2, ip ? 1 : 0, scratch, db, ep.dense_cap, od, oi,
                                  kc, sms, o.scan_event_start, o.scan_event_stop, st);
        if (ds != PDX_OK) return ds;
        PDX_TRY(mark(4));
        PDX_TRY(mark(5));
        return PDX_OK;
    }
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char *p = scratch + off;
        off += rup(bytes);
        return p;
    };
    float *tau = reinterpret_cast<float *>(take((size_t)nq * 4));
    uint64_t *cand = reinterpret_cast<uint64_t *>(take((size_t)nq * ep.nslots * k * 8));
    uint64_t *topk = reinterpret_cast<uint64_t *>(take((size_t)nq * k * 8));
    uint64_t *refined = reinterpret_cast<uint64_t *>(take((size_t)nq * k * 8));
    uint64_t *final_keys = reinterpret_cast<uint64_t *>(take((size_t)nq * k * 8));
    unsigned long long *counters = reinterpret_cast<unsigned long long *>(take(C_COUNT * 8));
    int *work = reinterpret_cast<int *>(take(8));
    uint16_t *qorder = ep.op.rows ? reinterpret_cast<uint16_t *>(take(ep.op.bytes)) : nullptr;
    float *pool = reinterpret_cast<float *>(take((size_t)nq * kPoolCap * 4));
    int32_t *pool_cnt = reinterpret_cast<int32_t *>(take((size_t)nq * 4));
    uint64_t *skeys = ep.start ? reinterpret_cast<uint64_t *>(take((size_t)nq * ep.Lstart * 8)) : nullptr;
    uint64_t *stopk = ep.start ? reinterpret_cast<uint64_t *>(take((size_t)nq * k * 8)) : nullptr;
    uint64_t *sc_keys = ep.start_clusters ? reinterpret_cast<uint64_t *>(take((size_t)nq * ep.sc_ld * 8)) : nullptr;
    uint64_t *sc_near = ep.start_clusters ? reinterpret_cast<uint64_t *>(take((size_t)nq * ep.sc_probe * 8)) : nullptr;
    uint64_t *sc_mkeys =
        ep.start_clusters ? reinterpret_cast<uint64_t *>(take((size_t)nq * ep.sc_probe * ix->sc_m * 8)) : nullptr;
    unsigned char *mlp_ws = ep.mlp_bytes ? take(ep.mlp_bytes) : nullptr;
    float *tau_in = o.tau_init ? reinterpret_cast<float *>(take((size_t)nq * 4)) : nullptr;
    uint64_t *sel_compact =
        nq <= kSplitSelectRows ? reinterpret_cast<uint64_t *>(take((size_t)nq * kSplitSelectCap * 8)) : nullptr;
    int32_t *sel_counts = nq <= kSplitSelectRows ? reinterpret_cast<int32_t *>(take((size_t)nq * 4)) : nullptr;
    float *cs_q = pl.pruner == PDX_PRUNE_CS_IP
                      ? reinterpret_cast<float *>(take((size_t)nq * (ix->cs_nchk + 1) * 2 * 4))
                      : nullptr;
    if (off > ep.bytes) {
        set_error("internal error: exact-search scratch layout exceeds its plan");
        return PDX_ERR_CUDA;
    }
    const float *scores = nullptr;
    bool learned_done = false;
    if (ep.op.mode == 2) {
        // learned order: each query's nearest centroid, network input [q; c],
        // BF16 inference into per-dimension scores
        const int hidden = o.mlp->hidden;
        unsigned char *mp = mlp_ws;
        uint64_t *ckeys = reinterpret_cast<uint64_t *>(mp);
        mp += rup((size_t)nq * ep.mlp_Lc * 8);
        uint64_t *nearest = reinterpret_cast<uint64_t *>(mp);
        mp += rup((size_t)nq * 8);
        float *u = reinterpret_cast<float *>(mp);
        mp += rup((size_t)nq * 2 * d * 4);
        float *zb = reinterpret_cast<float *>(mp);
        mp += rup((size_t)nq * hidden * 4);
        float *yb = reinterpret_cast<float *>(mp);
        PDX_TRY(launch_fill_u64(ckeys, kEmptyKey, nq * ep.mlp_Lc, st));
        PDX_TRY(launch_dense_keys_rows(qd, nq, o.mlp_centroids, o.mlp_ncentroids, d, ep.mlp_Lc, ckeys, st));
        PDX_TRY(launch_select_k(ckeys, nq, ep.mlp_Lc, 1, nearest, st));
        if (hidden % 2 == 0) {
            // inputs, both layers, the score and the sort in one launch
            PDX_TRY(mlp_order(o.mlp, qd, nq, o.mlp_centroids, nearest, ix->cmean, qorder, st));
            learned_done = true;
        } else {
            PDX_TRY(launch_mlp_inputs(qd, nq, d, o.mlp_centroids, nearest, u, st));
            PDX_TRY(mlp_scores(o.mlp, u, nq, zb, yb, st));
            scores = yb;
        }
    }
    if (cs_q)  // the query's whole and unvisited squared norms at the check points
        PDX_TRY(launch_bsa_qaux(qd, nq, d, nullptr, ix->cs_chk, ix->cs_nchk + 1, cs_q, st));
    if (ep.op.rows && !learned_done)  // query preprocessing (Sec. 5): PDX-BOND visit orders
        PDX_TRY(launch_order(qd, ep.op.rows, d, ep.op.per_part ? ix->means : ix->cmean, ep.op.per_part, nullptr,
                             ep.op.mode, std::max(1, (int)o.zone_dims), scores, qorder, st));
    PDX_TRY(mark(1));
    PDX_TRY(mark(2));
    PDX_TRY(launch_fill_u32(reinterpret_cast<uint32_t *>(tau), 0xff800000u, nq, st));  // ordered +inf
    PDX_TRY(cudaMemsetAsync(counters, 0, C_COUNT * 8, st));
    PDX_TRY(cudaMemsetAsync(work, 0, 8, st));
    const bool use_pool = pl.pruner != PDX_PRUNE_NONE && !o.tau_fixed;
    if (use_pool) {
        PDX_TRY(launch_fill_u32(reinterpret_cast<uint32_t *>(pool), 0x7f800000u, nq * kPoolCap, st));  // +inf
        PDX_TRY(cudaMemsetAsync(pool_cnt, 0, (size_t)nq * 4, st));
    }
    // kernels accumulate into the caller's device stats when given, else into scratch
    unsigned long long *kc = o.stats_device ? reinterpret_cast<unsigned long long *>(o.stats_device) : counters;
    if (counters_out) *counters_out = kc;
    if (ep.start_clusters) {
        // START (Sec. 4) from the query's kStartProbe nearest start clusters:
        // exact distances to their members give every query an initial
        // k-th-best threshold of real vectors near it
        const int P = ep.sc_probe, M = ix->sc_m;
        PDX_TRY(launch_dense_keys_rows(qd, nq, ix->sc_cent, ix->sc_c, d, ep.sc_ld, sc_keys, st));
        PDX_TRY(launch_select_k(sc_keys, nq, ep.sc_ld, P, sc_near, st));
        PDX_TRY(launch_member_keys(qd, nq, d, ix->xnary, ix->data, ix->slot_of, sc_near, P, ix->sc_members, M, sc_mkeys,
                                   st));
        PDX_TRY(launch_select_k(sc_mkeys, nq, (int64_t)P * M, k, stopk, st));
        PDX_TRY(launch_tau_from_keys(stopk, nq, k, tau, st));
        PDX_TRY(launch_add_u64(kc + C_START, (unsigned long long)nq * ((uint64_t)ix->sc_c + (uint64_t)P * M) * d, st));
    } else if (ep.start) {
        // START (Sec. 4): exact distances of the first start_vectors stored
        // vectors give every query an initial k-th-best threshold
        if (ix->storage == PDX_F32) {
            PDX_TRY(launch_dense_keys(qd, nq, ix->data, ix->ids, d, ep.start_blk, pl.metric, skeys, st));
        } else {  // exact FP32 from the vectors' FP32 copy, so tau is a real k-th distance
            const int32_t rows = (int32_t)std::min<int64_t>(ix->n, ep.Lstart);
            PDX_TRY(launch_fill_u64(skeys, kEmptyKey, nq * ep.Lstart, st));
            PDX_TRY(launch_dense_keys_rows(qd, nq, ix->xnary, rows, d, ep.Lstart, skeys, st));
        }
        PDX_TRY(launch_select_k(skeys, nq, ep.Lstart, k, stopk, st));
        PDX_TRY(launch_tau_from_keys(stopk, nq, k, tau, st));
        PDX_TRY(launch_add_u64(kc + C_START, (unsigned long long)nq * ep.Lstart * d, st));
    }
    if (tau_in) {  // the caller's initial thresholds
        PDX_TRY(cudaMemcpyAsync(tau_in, o.tau_init, (size_t)nq * 4, cudaMemcpyDefault, st));
        PDX_TRY(launch_tau_min(tau, tau_in, nq, st));
    }
    PDX_TRY(mark(3));
    ScanParams p;
    std::memset(&p, 0, sizeof p);
    p.data = ix->data;
    p.data_lp = ix->data_lp;
    p.storage = (int)ix->storage;
    p.scale = ix->scale;
    p.xnary = ix->xnary;
    p.ids = ix->ids;
    p.blk_cnt = ix->blk_cnt;
    p.part_blk = ix->part_blk;
    p.d = d;
    p.q = qd;
    p.qrows = qd;
    p.nq = nq;
    p.means = ix->means;
    p.probes = nullptr;
    p.nslots = ep.nslots;
    p.part0 = 0;
    p.chunks_per_part = ep.chunks;
    p.blocks_per_item = ep.bpi;
    p.k = k;
    p.tau = tau;
    p.cand = cand;
    p.counters = kc;
    p.work_counter = work;
    p.nitems = nq * (int64_t)ep.nslots;
    p.first_step = (int)o.first_step;
    p.sel_count = std::min(kMaxSurv, (int)std::ceil(o.selection_threshold * kBlock) - 1);
    if (p.sel_count < 0) p.sel_count = 0;
    p.zone_dims = (int)o.zone_dims;
    p.order = (int)o.order;
    p.ctas_per_sm = (int)o.ctas_per_sm;
    p.gamma = (float)d * 1.1920929e-7f;  // D * 2^-23
    p.eps0 = o.eps0;
    p.bsa_m = o.bsa_m;
    p.qorder = qorder;
    p.qorder_per_part = ep.op.per_part;
    p.pool = use_pool ? pool : nullptr;
    p.pool_cnt = pool_cnt;
    p.tau_fixed = o.tau_fixed ? 1 : 0;
    p.rows_vec4 = rows_vec4(ix, p.qrows);
    if (cs_q) {
        p.qaux = cs_q;
        p.resid = ix->cs_resid;
        p.nchk = ix->cs_nchk;
    }
    p.fin_log = o.finished_log;
    p.fin_count = o.finished_count;
    p.fin_cap = o.finished_cap;
    if (o.scan_event_start) PDX_TRY(cudaEventRecord(static_cast<cudaEvent_t>(o.scan_event_start), st));
    PDX_TRY(launch_scan(pl.pruner, pl.metric, p, sms, st));
    if (o.scan_event_stop) PDX_TRY(cudaEventRecord(static_cast<cudaEvent_t>(o.scan_event_stop), st));
    PDX_TRY(mark(4));
    PDX_TRY(launch_select_k_tau(cand, nq, (int64_t)ep.nslots * k, k, tau, p.gamma, topk, st, sel_compact, sel_counts));
    // canonical distances: from the contiguous rows when the index keeps them
    // (same lanes, order and reduction as from the blocks, so the same bits)
    if (ix->xnary && ix->metric != PDX_L1)
        PDX_TRY(launch_refine_rows(topk, nq, k, qd, d, ix->xnary, ix->metric, refined, st));
    else
        PDX_TRY(launch_refine(topk, nq, k, qd, d, ix->data, ix->slot_of, ix->metric, refined, st));
    PDX_TRY(launch_select_k(refined, nq, k, k, final_keys, st));
    PDX_TRY(launch_write_out(final_keys, nq, k, pl.out_mode, qd, d, od, oi, st));
    PDX_TRY(mark(5));
    return PDX_OK;
}

PhaseEvents::PhaseEvents() {
    for (auto &x : e) x = nullptr;
    ok = true;
    for (auto &x : e)
        if (cudaEventCreate(&x) != cudaSuccess) ok = false;
}
PhaseEvents::~PhaseEvents() {
    for (auto &x : e)
        if (x) cudaEventDestroy(x);
}
// Call after the stream has been synchronised.
void PhaseEvents::fill(pdx_search_stats *so) const {
    for (int i = 0; i < 5; ++i) {
        float ms = 0.f;
        so->phase_ns[i] = (ok && cudaEventElapsedTime(&ms, e[i], e[i + 1]) == cudaSuccess && ms > 0.f)
                              ? (uint64_t)((double)ms * 1e6 + 0.5)
                              : 0;
    }
}

void fill_stats(pdx_search_stats *so, const unsigned long long *c, const pdx_index *ix) {
    std::memset(so, 0, sizeof *so);
    so->values_visited = c[C_VALUES];
    so->vectors_scanned = c[C_SCANNED];
    so->vectors_pruned = c[C_PRUNED];
    so->prune_phase_blocks = c[C_PRUNE_BLOCKS];
    so->candidates = c[C_CANDIDATES];
    so->work_items = c[C_ITEMS];
    so->start_values = c[C_START];
    so->dense_fallbacks = c[C_DENSE_FALLBACK];
    so->bytes_logical = c[C_VALUES] * elem_size(ix->storage) + c[C_START] * 4ull +
                        (ix->storage == PDX_F32 ? 0ull : c[C_CANDIDATES] * (uint64_t)ix->d * 4ull);
}

pdx_status exact_check(const pdx_index *ix, const float *q, int64_t nq, int32_t k, const pdx_search_opts *opts,
                       float *out_dist, int64_t *out_idx, pdx_search_opts *o, SearchPlan *pl, const char *fn) {
    pdx_status s = check_search_args(ix, q, nq, k, opts, out_dist, out_idx, o, fn);
    if (s != PDX_OK) return s;
    if (ix->is_ivf) {
        set_error("%s: index was built by pdx_ivf_build", fn);
        return PDX_ERR_ARG;
    }
    if (o->pruner != PDX_PRUNE_NONE && o->pruner != PDX_PRUNE_BOND && o->pruner != PDX_PRUNE_CS_IP) {
        set_error("%s: only NONE, BOND or CS_IP keep the search exact", fn);
        return PDX_ERR_ARG;
    }
    if (o->pruner == PDX_PRUNE_CS_IP) {
        if (ix->cs_first_step <= 0) {
            set_error("%s: PDX_PRUNE_CS_IP needs an inner-product index built with cs_first_step", fn);
            return PDX_ERR_UNSUPPORTED;
        }
        // the stored norms fix the fetch schedule (the check points)
        o->first_step = (uint32_t)ix->cs_first_step;
    }
    if (q && (q == out_dist || (const void *)q == (const void *)out_idx)) {
        set_error("%s: outputs alias the queries", fn);
        return PDX_ERR_ARG;
    }
    return plan_metric(ix, o->pruner, pl, fn);
}

}  // namespace pdx

extern "C" pdx_status pdx_search_exact(const pdx_index *ix, const float *q, int64_t nq, int32_t k,
                                       const pdx_search_opts *opts, float *out_dist, int64_t *out_idx,
                                       void *stream) {
    const char *fn = "pdx_search_exact";
    pdx_search_opts o;
    SearchPlan pl;
    pdx_status s = exact_check(ix, q, nq, k, opts, out_dist, out_idx, &o, &pl, fn);
    if (s != PDX_OK) return s;
    if (nq == 0) return PDX_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int d = ix->d;
    const bool q_dev = is_device_ptr(q);
    const bool o_dev = is_device_ptr(out_dist) && is_device_ptr(out_idx);
    if (is_device_ptr(out_dist) != is_device_ptr(out_idx)) {
        set_error("%s: out_dist and out_idx must both be host or both be device memory", fn);
        return PDX_ERR_ARG;
    }
    const int sms = num_sms();
    ExactPlan ep;
    s = exact_plan(ix, nq, k, o, pl, sms, &ep);
    if (s != PDX_OK) return s;
    Scratch scr(st);
    size_t need = ep.bytes;
    if (!q_dev) need += rup((size_t)nq * d * 4);
    if (!o_dev) need += rup((size_t)nq * k * 4) + rup((size_t)nq * k * 8);
    PDX_TRY(scr.reserve(need));
    unsigned char *work = scr.take<unsigned char>(ep.bytes);
    const float *qd = q;
    float *qs = q_dev ? nullptr : scr.take<float>((size_t)nq * d);
    float *od = out_dist;
    int64_t *oi = out_idx;
    if (!o_dev) {
        od = scr.take<float>((size_t)nq * k);
        oi = scr.take<int64_t>((size_t)nq * k);
    }
    PDX_CHECK_SCRATCH(scr);
    if (!q_dev) {
        PDX_TRY(cudaMemcpyAsync(qs, q, (size_t)nq * d * 4, cudaMemcpyHostToDevice, st));
        qd = qs;
    }
    unsigned long long *kc = nullptr;
    std::unique_ptr<PhaseEvents> ph;
    if (o.stats_out) {
        ph.reset(new (std::nothrow) PhaseEvents());
        if (ph && !ph->ok) ph.reset();
    }
    s = exact_run(ix, qd, nq, k, o, pl, ep, work, od, oi, &kc, sms, st, ph.get());
    if (s != PDX_OK) return s;
    if (!o_dev) {
        PDX_TRY(cudaMemcpyAsync(out_dist, od, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, st));
        PDX_TRY(cudaMemcpyAsync(out_idx, oi, (size_t)nq * k * 8, cudaMemcpyDeviceToHost, st));
    }
    if (o.stats_out) {
        unsigned long long c[C_COUNT];
        PDX_TRY(cudaMemcpyAsync(c, kc, sizeof c, cudaMemcpyDeviceToHost, st));
        PDX_TRY(cudaStreamSynchronize(st));
        fill_stats(o.stats_out, c, ix);
        if (ph) ph->fill(o.stats_out);
    }
    if (!o_dev) PDX_TRY(cudaStreamSynchronize(st));
    return PDX_OK;
}

namespace pdx {

// splitmix64: picks the initial k-means centroids from the seed
static uint64_t splitmix64(uint64_t &st) {
    uint64_t z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ADSampling's random orthogonal transformation (Sec. 2.3), drawn from a seed:
// a d x d matrix of standard normal values, its QR factorisation in FP64 by
// Householder reflections, and Q with each column multiplied by the sign of
// R's diagonal entry, which makes Q Haar-distributed over the orthogonal
// group. Normal values: Box-Muller on uniform doubles from a splitmix64
// counter stream (two 53-bit uniforms per value).
static void random_orthogonal(int d, uint64_t seed, std::vector<float> &out) {
    const size_t dd = (size_t)d;
    std::vector<double> A(dd * dd);  // row-major A[i][j]
    uint64_t st = seed ^ 0x5D58A6E1C4B3F207ull;
    const double two_pi = 6.283185307179586476925;
    for (size_t e = 0; e < dd * dd; ++e) {
        const double u1 = 1.0 - (double)(splitmix64(st) >> 11) * 0x1.0p-53;  // (0, 1]
        const double u2 = (double)(splitmix64(st) >> 11) * 0x1.0p-53;        // [0, 1)
        A[e] = std::sqrt(-2.0 * std::log(u1)) * std::cos(two_pi * u2);
    }
    // Householder: for column k, v = x - alpha e_1 with alpha = -sign(x_0) ||x||
    // (so R_kk = alpha), reflecting rows k.. of the trailing columns.
    std::vector<double> V(dd * dd, 0.0), w(dd);
    std::vector<double> rdiag(dd);
    for (int k = 0; k < d; ++k) {
        double nrm2 = 0.0;
        for (int i = k; i < d; ++i) nrm2 += A[(size_t)i * dd + k] * A[(size_t)i * dd + k];
        const double x0 = A[(size_t)k * dd + k];
        const double alpha = (x0 >= 0.0 ? -1.0 : 1.0) * std::sqrt(nrm2);
        rdiag[(size_t)k] = alpha;
        double *v = &V[(size_t)k * dd];  // v over rows k..d-1
        double vn2 = 0.0;
        for (int i = k; i < d; ++i) {
            v[i] = A[(size_t)i * dd + k] - (i == k ? alpha : 0.0);
            vn2 += v[i] * v[i];
        }
        if (vn2 == 0.0) continue;  // column already reduced: H_k = I
        const double inv = 1.0 / std::sqrt(vn2);
        for (int i = k; i < d; ++i) v[i] *= inv;
        // A[k:, k:] -= 2 v (v^T A[k:, k:])
        std::fill(w.begin() + k, w.end(), 0.0);
        for (int i = k; i < d; ++i) {
            const double vi = v[i];
            const double *row = &A[(size_t)i * dd];
            for (int j = k; j < d; ++j) w[(size_t)j] += vi * row[j];
        }
        for (int i = k; i < d; ++i) {
            const double vi2 = 2.0 * v[i];
            double *row = &A[(size_t)i * dd];
            for (int j = k; j < d; ++j) row[j] -= vi2 * w[(size_t)j];
        }
    }
    // Q = H_0 H_1 ... H_{d-1}: applied to I from the last reflection back
    std::vector<double> Q(dd * dd, 0.0);
    for (int i = 0; i < d; ++i) Q[(size_t)i * dd + i] = 1.0;
    for (int k = d - 1; k >= 0; --k) {
        const double *v = &V[(size_t)k * dd];
        bool zero = true;
        for (int i = k; i < d && zero; ++i) zero = (v[i] == 0.0);
        if (zero) continue;
        std::fill(w.begin(), w.end(), 0.0);
        for (int i = k; i < d; ++i) {
            const double vi = v[i];
            const double *row = &Q[(size_t)i * dd];
            for (int j = 0; j < d; ++j) w[(size_t)j] += vi * row[j];
        }
        for (int i = k; i < d; ++i) {
            const double vi2 = 2.0 * v[i];
            double *row = &Q[(size_t)i * dd];
            for (int j = 0; j < d; ++j) row[j] -= vi2 * w[(size_t)j];
        }
    }
    out.assign(dd * dd, 0.f);
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            const double sgn = rdiag[(size_t)j] < 0.0 ? -1.0 : 1.0;
            out[(size_t)i * dd + j] = (float)(Q[(size_t)i * dd + j] * sgn);
        }
}

// PCA of the (sample of the) vectors for BSA: rot rows = eigenvectors of the
// covariance by decreasing eigenvalue (ties: lower index), shift = mean,
// var = eigenvalues (clamped at 0).
static pdx_status build_pca(pdx_index *ix, const float *xd, int64_t m, cudaStream_t st) {
    const int d = ix->d;
    Scratch scr(st);
    const size_t nwork = (size_t)d * d * 2 + 2 * (size_t)(d + 1) + (size_t)(d + 2);
    size_t need = rup((size_t)d * 8) + 2 * rup((size_t)d * d * 8) + rup(nwork * 8);
    PDX_TRY(scr.reserve(need));
    double *sum = scr.take<double>(d);
    double *A = scr.take<double>((size_t)d * d);
    double *V = scr.take<double>((size_t)d * d);
    double *work = scr.take<double>(nwork);
    PDX_CHECK_SCRATCH(scr);
    PDX_TRY(launch_column_stats(xd, m, d, sum, A, st));
    std::vector<double> hs(d), hA((size_t)d * d);
    PDX_TRY(cudaMemcpyAsync(hs.data(), sum, (size_t)d * 8, cudaMemcpyDeviceToHost, st));
    PDX_TRY(cudaMemcpyAsync(hA.data(), A, (size_t)d * d * 8, cudaMemcpyDeviceToHost, st));
    PDX_TRY(cudaStreamSynchronize(st));
    std::vector<double> mean(d);
    for (int j = 0; j < d; ++j) mean[j] = hs[j] / (double)m;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) hA[(size_t)i * d + j] = hA[(size_t)i * d + j] / (double)m - mean[i] * mean[j];
    std::vector<double> eye((size_t)d * d, 0.0);
    for (int i = 0; i < d; ++i) eye[(size_t)i * d + i] = 1.0;
    PDX_TRY(cudaMemcpyAsync(A, hA.data(), hA.size() * 8, cudaMemcpyHostToDevice, st));
    PDX_TRY(cudaMemcpyAsync(V, eye.data(), eye.size() * 8, cudaMemcpyHostToDevice, st));
    PDX_TRY(jacobi_eigen(A, V, d, work, 10, st));
    std::vector<double> hV((size_t)d * d);
    PDX_TRY(cudaMemcpyAsync(hA.data(), A, hA.size() * 8, cudaMemcpyDeviceToHost, st));
    PDX_TRY(cudaMemcpyAsync(hV.data(), V, hV.size() * 8, cudaMemcpyDeviceToHost, st));
    PDX_TRY(cudaStreamSynchronize(st));
    std::vector<int> order(d);
    for (int i = 0; i < d; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return hA[(size_t)a * d + a] > hA[(size_t)b * d + b]; });
    std::vector<float> rot((size_t)d * d), shift(d), var(d);
    for (int r = 0; r < d; ++r) {
        int c = order[r];
        for (int j = 0; j < d; ++j) rot[(size_t)r * d + j] = (float)hV[(size_t)j * d + c];
        var[r] = (float)std::max(0.0, hA[(size_t)c * d + c]);
    }
    for (int j = 0; j < d; ++j) shift[j] = (float)mean[j];
    PDX_TRY(dalloc(ix, &ix->rot, (size_t)d * d));
    PDX_TRY(dalloc(ix, &ix->shift, (size_t)d));
    PDX_TRY(dalloc(ix, &ix->pca_var, (size_t)d));
    PDX_TRY(cudaMemcpyAsync(ix->rot, rot.data(), rot.size() * 4, cudaMemcpyHostToDevice, st));
    PDX_TRY(cudaMemcpyAsync(ix->shift, shift.data(), shift.size() * 4, cudaMemcpyHostToDevice, st));
    PDX_TRY(cudaMemcpyAsync(ix->pca_var, var.data(), var.size() * 4, cudaMemcpyHostToDevice, st));
    PDX_TRY(cudaStreamSynchronize(st));
    return PDX_OK;
}

static pdx_status ivf_build_impl(pdx_index *ix, const float *x, const pdx_ivf_opts &o, cudaStream_t st) {
    const int64_t n = ix->n;
    const int d = ix->d;
    const int nlist = (int)o.nlist;
    Scratch scr(st);
    const bool xdev = is_device_ptr(x);
    const bool tr = o.transform != PDX_PRUNE_NONE;
    const int64_t mtrain = (o.kmeans_sample > 0 && (int64_t)o.kmeans_sample < n) ? (int64_t)o.kmeans_sample : n;
    size_t need = (xdev ? 0 : rup((size_t)n * d * 4)) + (tr ? rup((size_t)n * d * 4) : 0) +
                  rup((size_t)nlist * d * 4) + rup((size_t)nlist * 4) + rup((size_t)n * 4) + rup((size_t)nlist * d * 4);
    PDX_TRY(scr.reserve(need));
    const float *xd = x;
    if (!xdev) {
        float *t = scr.take<float>((size_t)n * d);
        PDX_CHECK_SCRATCH(scr);
        PDX_TRY(cudaMemcpyAsync(t, x, (size_t)n * d * 4, cudaMemcpyHostToDevice, st));
        xd = t;
    }
    // Sec. 2.3: ADSampling stores R x (random orthogonal R, given by the
    // caller); BSA stores the PCA projection W^T (x - mean)
    const float *xt = xd;
    if (tr) {
        float *t = scr.take<float>((size_t)n * d);
        PDX_CHECK_SCRATCH(scr);
        if (o.transform == PDX_PRUNE_ADSAMPLING) {
            PDX_TRY(dalloc(ix, &ix->rot, (size_t)d * d));
            if (o.rotation) {
                PDX_TRY(cudaMemcpyAsync(ix->rot, o.rotation, (size_t)d * d * 4, cudaMemcpyDefault, st));
            } else {
                std::vector<float> P;
                random_orthogonal(d, o.rotation_seed, P);
                PDX_TRY(cudaMemcpyAsync(ix->rot, P.data(), P.size() * 4, cudaMemcpyHostToDevice, st));
                PDX_TRY(cudaStreamSynchronize(st));
            }
            PDX_TRY(launch_transform(xd, n, d, ix->rot, nullptr, t, st));
        } else {
            pdx_status s = build_pca(ix, xd, std::min<int64_t>(n, 262144), st);
            if (s != PDX_OK) return s;
            PDX_TRY(launch_transform(xd, n, d, ix->rot, ix->shift, t, st));
        }
        xt = t;
    }
    // Lloyd's k-means (Sec. 2.1) on the first mtrain transformed vectors
    float *sums = scr.take<float>((size_t)nlist * d);
    int32_t *counts = scr.take<int32_t>((size_t)nlist);
    int32_t *tassign = scr.take<int32_t>((size_t)n);
    float *cinit = scr.take<float>((size_t)nlist * d);
    PDX_CHECK_SCRATCH(scr);
    PDX_TRY(dalloc(ix, &ix->centroids, (size_t)nlist * d));
    if (o.init_centroids) {
        PDX_TRY(cudaMemcpyAsync(cinit, o.init_centroids, (size_t)nlist * d * 4, cudaMemcpyDefault, st));
        if (tr)
            PDX_TRY(launch_transform(cinit, nlist, d, ix->rot, ix->shift, ix->centroids, st));
        else
            PDX_TRY(cudaMemcpyAsync(ix->centroids, cinit, (size_t)nlist * d * 4, cudaMemcpyDeviceToDevice, st));
    } else {
        // nlist distinct training vectors chosen by a seeded partial shuffle
        std::vector<int64_t> pick((size_t)mtrain);
        for (int64_t i = 0; i < mtrain; ++i) pick[(size_t)i] = i;
        uint64_t sm = o.seed;
        for (int c = 0; c < nlist; ++c) {
            int64_t j = c + (int64_t)(splitmix64(sm) % (uint64_t)(mtrain - c));
            std::swap(pick[(size_t)c], pick[(size_t)j]);
            PDX_TRY(cudaMemcpyAsync(ix->centroids + (size_t)c * d, xt + (size_t)pick[(size_t)c] * d, (size_t)d * 4,
                                    cudaMemcpyDeviceToDevice, st));
        }
    }
    for (uint32_t it = 0; it < o.kmeans_iters; ++it) {
        PDX_TRY(launch_nearest_centroids(xt, mtrain, d, ix->centroids, nullptr, nlist, tassign, nullptr, st));
        PDX_TRY(launch_kmeans_update(xt, mtrain, d, tassign, nlist, sums, counts, ix->centroids, st));
    }
    PDX_TRY(dalloc(ix, &ix->assign, (size_t)n));
    PDX_TRY(launch_nearest_centroids(xt, n, d, ix->centroids, nullptr, nlist, ix->assign, nullptr, st));
    // buckets = PDXearch blocks (Fig. 2): vectors grouped by bucket, id order inside
    std::vector<int32_t> ha((size_t)n);
    PDX_TRY(cudaMemcpyAsync(ha.data(), ix->assign, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
    PDX_TRY(cudaStreamSynchronize(st));
    std::vector<int64_t> part_row((size_t)nlist + 1, 0);
    for (int64_t i = 0; i < n; ++i) part_row[(size_t)ha[(size_t)i] + 1] += 1;
    for (int c = 0; c < nlist; ++c) part_row[(size_t)c + 1] += part_row[(size_t)c];
    std::vector<int64_t> fill(part_row.begin(), part_row.end() - 1);
    std::vector<int32_t> rows((size_t)n);
    for (int64_t i = 0; i < n; ++i) rows[(size_t)fill[(size_t)ha[(size_t)i]]++] = (int32_t)i;
    pdx_status s = layout_parts(ix, xt, rows, part_row, st);
    if (s != PDX_OK) return s;
    // per-bucket variances (the fused pruner's expected contributions)
    PDX_TRY(dalloc(ix, &ix->vars, (size_t)nlist * d));
    PDX_TRY(launch_part_vars(ix->data, ix->blk_cnt, ix->part_blk, nlist, d, ix->means, ix->vars, st));
    // centroids in PDX layout too (Sec. 6.4: the bucket search uses the PDX kernel)
    ix->c_nblocks = (nlist + kBlock - 1) / kBlock;
    std::vector<int32_t> cids((size_t)ix->c_nblocks * kBlock, -1);
    for (int c = 0; c < nlist; ++c) cids[(size_t)c] = c;
    PDX_TRY(dalloc(ix, &ix->cids, cids.size()));
    PDX_TRY(dalloc(ix, &ix->cdata, (size_t)ix->c_nblocks * d * kBlock));
    PDX_TRY(cudaMemcpyAsync(ix->cids, cids.data(), cids.size() * 4, cudaMemcpyHostToDevice, st));
    PDX_TRY(launch_to_pdx(ix->centroids, d, ix->cids, ix->c_nblocks, ix->cdata, st));
    if (o.transform == PDX_PRUNE_BSA) {
        std::vector<int32_t> chk = check_points(d, ix->bsa_first_step);
        ix->bsa_nchk = (int)chk.size();
        if (ix->bsa_nchk > 0) {
            PDX_TRY(dalloc(ix, &ix->chk, chk.size()));
            PDX_TRY(dalloc(ix, &ix->resid, (size_t)ix->nblocks * ix->bsa_nchk * kBlock));
            PDX_TRY(cudaMemcpyAsync(ix->chk, chk.data(), chk.size() * 4, cudaMemcpyHostToDevice, st));
            PDX_TRY(launch_bsa_resid(ix->data, ix->blk_cnt, ix->nblocks, d, ix->chk, ix->bsa_nchk, ix->resid, st));
        }
    }
    PDX_TRY(cudaStreamSynchronize(st));
    // rows by id: the original vectors, so that full distances (row finish,
    // rerank, canonical refine) carry no rounding of the transform
    if (ix->storage != PDX_F32) return finish_low_precision(ix, xt, xd, st);
    if (o.base.keep_rows) return keep_rows(ix, xd, st);
    return PDX_OK;
}

}  // namespace pdx

extern "C" pdx_status pdx_ivf_build(const float *x, int64_t n, int32_t d, const pdx_ivf_opts *opts, void *stream,
                                    pdx_index **out) {
    if (out) *out = nullptr;
    if (!x || !out || !opts) {
        set_error("pdx_ivf_build: NULL x, opts or out");
        return PDX_ERR_ARG;
    }
    if (opts->struct_size < sizeof(pdx_ivf_opts)) {
        set_error("pdx_ivf_build: opts->struct_size %u < %zu", opts->struct_size, sizeof(pdx_ivf_opts));
        return PDX_ERR_ARG;
    }
    const pdx_ivf_opts o = *opts;
    if (n < 1 || n >= (int64_t)1 << 31 || d < 1 || d > kMaxD || o.nlist < 1 || (int64_t)o.nlist > n) {
        set_error("pdx_ivf_build: n=%lld d=%d nlist=%u out of range", (long long)n, d, o.nlist);
        return PDX_ERR_ARG;
    }
    if (!valid_metric(o.base.metric) || o.transform < PDX_PRUNE_NONE || o.transform > PDX_PRUNE_BSA ||
        o.transform == PDX_PRUNE_BOND) {
        set_error("pdx_ivf_build: bad metric %d or transform %d", (int)o.base.metric, (int)o.transform);
        return PDX_ERR_ARG;
    }
    if (o.kmeans_sample != 0 && o.kmeans_sample < o.nlist) {
        set_error("pdx_ivf_build: kmeans_sample=%u must be 0 (all) or >= nlist=%u", o.kmeans_sample, o.nlist);
        return PDX_ERR_ARG;
    }
    if (o.base.storage != PDX_F32 && o.base.metric == PDX_L1) {
        set_error("pdx_ivf_build: low-precision storage supports L2 (and unit-norm IP) only");
        return PDX_ERR_UNSUPPORTED;
    }
    if (o.base.cs_first_step != 0) {
        set_error("pdx_ivf_build: cs_first_step (the Cauchy-Schwarz inner-product norms) is for exact indexes");
        return PDX_ERR_UNSUPPORTED;
    }
    if (o.transform != PDX_PRUNE_NONE && o.base.metric != PDX_L2) {
        set_error("pdx_ivf_build: ADSampling/BSA transforms are defined for L2 only");
        return PDX_ERR_UNSUPPORTED;
    }
    pdx_index *ix = new (std::nothrow) pdx_index();
    if (!ix) {
        set_error("host allocation failed");
        return PDX_ERR_OOM;
    }
    ix->n = n;
    ix->d = d;
    ix->metric = o.base.metric;
    ix->storage = o.base.storage;
    ix->is_ivf = 1;
    ix->transform = o.transform;
    cudaGetDevice(&ix->device);
    pdx_status s = ivf_build_impl(ix, x, o, static_cast<cudaStream_t>(stream));
    if (s != PDX_OK) {
        free_index(ix);
        return s;
    }
    *out = ix;
    return PDX_OK;
}

extern "C" pdx_status pdx_search_ivf(const pdx_index *ix, const float *q, int64_t nq, int32_t k, int32_t nprobe,
                                     const pdx_search_opts *opts, float *out_dist, int64_t *out_idx, void *stream) {
    const char *fn = "pdx_search_ivf";
    pdx_search_opts o;
    pdx_status s = check_search_args(ix, q, nq, k, opts, out_dist, out_idx, &o, fn);
    if (s != PDX_OK) return s;
    if (!ix->is_ivf) {
        set_error("%s: index was not built by pdx_ivf_build", fn);
        return PDX_ERR_ARG;
    }
    if (o.engine == PDX_ENGINE_TENSOR) {
        set_error("%s: the tensor-core engine serves exact indexes only", fn);
        return PDX_ERR_UNSUPPORTED;
    }
    if (nprobe < 1 || nprobe > ix->nparts || nprobe > 4096) {
        set_error("%s: nprobe=%d outside [1, min(nlist=%d, 4096)]", fn, nprobe, ix->nparts);
        return PDX_ERR_ARG;
    }
    if (o.pruner == PDX_PRUNE_CS_IP) {
        set_error("%s: PDX_PRUNE_CS_IP serves exact inner-product indexes only", fn);
        return PDX_ERR_UNSUPPORTED;
    }
    if (((o.pruner == PDX_PRUNE_ADSAMPLING || o.pruner == PDX_PRUNE_ADS_BOND) &&
         ix->transform != PDX_PRUNE_ADSAMPLING) ||
        (o.pruner == PDX_PRUNE_BSA && ix->transform != PDX_PRUNE_BSA)) {
        set_error("%s: pruner %d needs an index built with that transform", fn, (int)o.pruner);
        return PDX_ERR_ARG;
    }
    // BSA's residual norms were stored at the check points of one fetch
    // schedule: a BSA search always uses that schedule
    if (o.pruner == PDX_PRUNE_BSA) o.first_step = (uint32_t)ix->bsa_first_step;
    if (q && (q == out_dist || (const void *)q == (const void *)out_idx)) {
        set_error("%s: outputs alias the queries", fn);
        return PDX_ERR_ARG;
    }
    SearchPlan pl;
    s = plan_metric(ix, o.pruner, &pl, fn);
    if (s != PDX_OK) return s;
    if (nq == 0) return PDX_OK;
    if (is_device_ptr(out_dist) != is_device_ptr(out_idx)) {
        set_error("%s: out_dist and out_idx must both be host or both be device memory", fn);
        return PDX_ERR_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int d = ix->d;
    const bool q_dev = is_device_ptr(q);
    const bool o_dev = is_device_ptr(out_dist);
    const bool tr = ix->transform != PDX_PRUNE_NONE;
    const int sms = num_sms();
    const int64_t Lc = (int64_t)ix->c_nblocks * kBlock;
    // check points: BSA's stored schedule, or (fused pruner) the search's own
    const std::vector<int32_t> adsb_chk =
        o.pruner == PDX_PRUNE_ADS_BOND ? check_points(d, (int)o.first_step) : std::vector<int32_t>();
    if ((int)adsb_chk.size() > kMaxChecks) {
        set_error("%s: first_step=%u gives %zu check points (at most %d)", fn, o.first_step, adsb_chk.size(),
                  kMaxChecks);
        return PDX_ERR_ARG;
    }
    const int nchk = (o.pruner == PDX_PRUNE_BSA) ? ix->bsa_nchk : (int)adsb_chk.size();
    int max_blk = 0;
    for (int p = 0; p < ix->nparts; ++p) max_blk = std::max(max_blk, ix->h_part_blk[p + 1] - ix->h_part_blk[p]);
    max_blk = std::max(1, max_blk);
    // work items: (query, probed bucket, group of its blocks). Buckets are
    // split into groups when the START launch (one nearest bucket per query)
    // would leave too few items to fill the GPU; every group of a query
    // shares its threshold through the query's candidate pool.
    int ivf_bpi = (int)o.blocks_per_item;
    if (ivf_bpi <= 0) {
        const int64_t target = (int64_t)sms * 64 * 3;
        const int64_t want = std::max<int64_t>(1, (target + nq - 1) / nq);
        const int ch = (int)std::min<int64_t>(max_blk, std::min<int64_t>(want, 8));
        ivf_bpi = (max_blk + ch - 1) / ch;
    }
    const int ivf_chunks = (max_blk + ivf_bpi - 1) / ivf_bpi;
    const int nslots = nprobe * ivf_chunks;
    const OrderPlan op = plan_orders(ix, o, pl.pruner, nq, nprobe);

    Scratch scr(st);
    size_t need = rup(op.bytes) + (q_dev ? 0 : rup((size_t)nq * d * 4)) + (tr ? rup((size_t)nq * d * 4) : 0) +
                  rup((size_t)nq * Lc * 8) + rup((size_t)nq * nprobe * 8) + rup((size_t)nq * nprobe * 4) +
                  rup((size_t)nq * 4) + rup((size_t)nq * nslots * k * 8) + 3 * rup((size_t)nq * k * 8) +
                  rup(C_COUNT * 8) + rup(16) + rup((size_t)nq * (nchk + 1) * 8) +
                  rup((size_t)nq * nprobe * std::max(1, nchk) * 4) + rup((size_t)kMaxChecks * 4) +
                  rup((size_t)nq * kPoolCap * 4) + rup((size_t)nq * 4) + (o.tau_init ? rup((size_t)nq * 4) : 0) +
                  (o_dev ? 0 : rup((size_t)nq * k * 4) + rup((size_t)nq * k * 8));
    PDX_TRY(scr.reserve(need));
    const float *qd = q;
    if (!q_dev) {
        float *t = scr.take<float>((size_t)nq * d);
        PDX_CHECK_SCRATCH(scr);
        PDX_TRY(cudaMemcpyAsync(t, q, (size_t)nq * d * 4, cudaMemcpyHostToDevice, st));
        qd = t;
    }
    const float *qt = qd;
    float *qt_buf = tr ? scr.take<float>((size_t)nq * d) : nullptr;
    uint64_t *pkeys = scr.take<uint64_t>((size_t)nq * Lc);
    uint64_t *ptopk = scr.take<uint64_t>((size_t)nq * nprobe);
    int32_t *probes = scr.take<int32_t>((size_t)nq * nprobe);
    float *tau = scr.take<float>((size_t)nq);
    uint64_t *cand = scr.take<uint64_t>((size_t)nq * nslots * k);
    uint64_t *topk = scr.take<uint64_t>((size_t)nq * k);
    uint64_t *refined = scr.take<uint64_t>((size_t)nq * k);
    uint64_t *final_keys = scr.take<uint64_t>((size_t)nq * k);
    unsigned long long *counters = scr.take<unsigned long long>(C_COUNT);
    int *work = scr.take<int>(4);
    float *qaux = scr.take<float>((size_t)nq * (nchk + 1) * 2);
    float *mass = scr.take<float>((size_t)nq * nprobe * std::max(1, nchk));
    int32_t *chk_dev = scr.take<int32_t>(kMaxChecks);
    uint16_t *qorder = op.rows ? scr.take<uint16_t>((size_t)op.rows * d) : nullptr;
    float *pool = scr.take<float>((size_t)nq * kPoolCap);
    int32_t *pool_cnt = scr.take<int32_t>((size_t)nq);
    float *tau_in = o.tau_init ? scr.take<float>((size_t)nq) : nullptr;
    float *od = out_dist;
    int64_t *oi = out_idx;
    if (!o_dev) {
        od = scr.take<float>((size_t)nq * k);
        oi = scr.take<int64_t>((size_t)nq * k);
    }
    PDX_CHECK_SCRATCH(scr);
    std::unique_ptr<PhaseEvents> ph;
    if (o.stats_out) {
        ph.reset(new (std::nothrow) PhaseEvents());
        if (ph && !ph->ok) ph.reset();
    }
    auto mark = [&](int i) -> cudaError_t { return ph ? cudaEventRecord(ph->e[i], st) : cudaSuccess; };
    PDX_TRY(mark(0));
    if (tr) {  // query preprocessing (Sec. 2.3): rotation or PCA projection
        PDX_TRY(launch_transform(qd, nq, d, ix->rot, ix->shift, qt_buf, st));
        qt = qt_buf;
    }
    if (nchk > 0 && o.pruner == PDX_PRUNE_BSA) PDX_TRY(launch_bsa_qaux(qt, nq, d, ix->pca_var, ix->chk, nchk, qaux, st));
    PDX_TRY(mark(1));
    // nearest buckets: PDX scan of the centroids, then the nprobe best per query
    PDX_TRY(launch_dense_keys(qt, nq, ix->cdata, ix->cids, d, ix->c_nblocks, PDX_L2, pkeys, st));
    PDX_TRY(launch_select_k(pkeys, nq, Lc, nprobe, ptopk, st));
    PDX_TRY(launch_keys_to_parts(ptopk, nq, nprobe, probes, st));
    if (op.rows)  // PDX-BOND visit orders against the probed buckets' (or the collection's) means
        PDX_TRY(launch_order(qt, op.rows, d, op.per_part ? ix->means : ix->cmean, op.per_part,
                             op.per_part ? probes : nullptr, op.mode, std::max(1, (int)o.zone_dims), nullptr, qorder,
                             st));
    if (o.pruner == PDX_PRUNE_ADS_BOND && nchk > 0) {  // F_q at every check point of every (query, bucket)
        PDX_TRY(cudaMemcpyAsync(chk_dev, adsb_chk.data(), adsb_chk.size() * 4, cudaMemcpyHostToDevice, st));
        PDX_TRY(launch_mass(qt, (int64_t)nq * nprobe, d, nprobe, probes, ix->means, ix->vars, qorder, chk_dev, nchk,
                            mass, st));
    }
    PDX_TRY(mark(2));
    PDX_TRY(launch_fill_u32(reinterpret_cast<uint32_t *>(tau), 0xff800000u, nq, st));
    PDX_TRY(cudaMemsetAsync(counters, 0, C_COUNT * 8, st));
    PDX_TRY(cudaMemsetAsync(work, 0, 16, st));
    const bool use_pool = pl.pruner != PDX_PRUNE_NONE && !o.tau_fixed;
    if (use_pool) {
        PDX_TRY(launch_fill_u32(reinterpret_cast<uint32_t *>(pool), 0x7f800000u, nq * kPoolCap, st));  // +inf
        PDX_TRY(cudaMemsetAsync(pool_cnt, 0, (size_t)nq * 4, st));
    }
    if (tau_in) {  // the caller's initial thresholds
        PDX_TRY(cudaMemcpyAsync(tau_in, o.tau_init, (size_t)nq * 4, cudaMemcpyDefault, st));
        PDX_TRY(launch_tau_min(tau, tau_in, nq, st));
    }
    unsigned long long *kc = o.stats_device ? reinterpret_cast<unsigned long long *>(o.stats_device) : counters;
    ScanParams p;
    std::memset(&p, 0, sizeof p);
    p.data = ix->data;
    p.data_lp = ix->data_lp;
    p.storage = (int)ix->storage;
    p.scale = ix->scale;
    p.xnary = ix->xnary;
    p.ids = ix->ids;
    p.blk_cnt = ix->blk_cnt;
    p.part_blk = ix->part_blk;
    p.d = d;
    p.q = qt;
    p.qrows = qd;  // the rows keep the original vectors
    p.nq = nq;
    p.means = ix->means;
    p.probes = probes;
    p.nslots = nslots;
    p.chunks_per_part = ivf_chunks;
    p.blocks_per_item = ivf_bpi;
    p.k = k;
    p.tau = tau;
    p.cand = cand;
    p.counters = kc;
    p.first_step = (int)o.first_step;
    p.sel_count = std::min(kMaxSurv, (int)std::ceil(o.selection_threshold * kBlock) - 1);
    if (p.sel_count < 0) p.sel_count = 0;
    p.zone_dims = (int)o.zone_dims;
    p.order = (int)o.order;
    p.ctas_per_sm = (int)o.ctas_per_sm;
    p.gamma = (float)d * 1.1920929e-7f;
    p.eps0 = o.eps0;
    p.bsa_m = o.bsa_m;
    p.qaux = (o.pruner == PDX_PRUNE_ADS_BOND) ? mass : qaux;
    p.resid = ix->resid;
    p.nchk = nchk;
    p.pool = use_pool ? pool : nullptr;
    p.pool_cnt = pool_cnt;
    p.qorder = qorder;
    p.qorder_per_part = op.per_part;
    p.tau_fixed = o.tau_fixed ? 1 : 0;
    p.rows_vec4 = rows_vec4(ix, p.qrows);
    p.fin_log = o.finished_log;
    p.fin_count = o.finished_count;
    p.fin_cap = o.finished_cap;
    if (o.scan_event_start) PDX_TRY(cudaEventRecord(static_cast<cudaEvent_t>(o.scan_event_start), st));
    // START (Sec. 4): every query's nearest bucket (slot 0, its block groups)
    // from tau = +inf, then WARMUP/PRUNE over the other buckets from the
    // thresholds it produced. When the START items fill at least two waves of
    // the GPU's warps, both run in one launch: items are numbered slot-major,
    // so the nearest buckets are handed out first and nearly all of them are
    // done before a later bucket starts, and no idle tail separates the phases
    // (1M x 960, 10,000 queries, nprobe 4: ADS 749k -> 786k queries/s; START's
    // time is then inside the scan phase). With fewer, a later bucket would
    // start before its query's START had a threshold: two launches.
    const bool one_launch = nq * (int64_t)ivf_chunks >= 2 * (int64_t)sms * 32;
    p.slot0 = 0;
    p.work_counter = work;
    if (one_launch) {
        p.nitems = nq * (int64_t)nprobe * ivf_chunks;
        PDX_TRY(mark(3));
        PDX_TRY(launch_scan(pl.pruner, pl.metric, p, sms, st));
    } else {
        p.nitems = nq * (int64_t)ivf_chunks;
        PDX_TRY(launch_scan(pl.pruner, pl.metric, p, sms, st));
        PDX_TRY(mark(3));
        if (nprobe > 1) {
            p.slot0 = ivf_chunks;
            p.nitems = nq * (int64_t)(nprobe - 1) * ivf_chunks;
            p.work_counter = work + 2;
            PDX_TRY(launch_scan(pl.pruner, pl.metric, p, sms, st));
        }
    }
    if (o.scan_event_stop) PDX_TRY(cudaEventRecord(static_cast<cudaEvent_t>(o.scan_event_stop), st));
    PDX_TRY(mark(4));
    PDX_TRY(launch_select_k(cand, nq, (int64_t)nslots * k, k, topk, st));
    // canonical distances from the rows (the original vectors, with the
    // untransformed queries) when the index keeps them
    if (ix->xnary && ix->metric != PDX_L1)
        PDX_TRY(launch_refine_rows(topk, nq, k, qd, d, ix->xnary, ix->metric, refined, st));
    else
        PDX_TRY(launch_refine(topk, nq, k, qt, d, ix->data, ix->slot_of, ix->metric, refined, st));
    PDX_TRY(launch_select_k(refined, nq, k, k, final_keys, st));
    PDX_TRY(launch_write_out(final_keys, nq, k, pl.out_mode, qd, d, od, oi, st));
    PDX_TRY(mark(5));
    if (!o_dev) {
        PDX_TRY(cudaMemcpyAsync(out_dist, od, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, st));
        PDX_TRY(cudaMemcpyAsync(out_idx, oi, (size_t)nq * k * 8, cudaMemcpyDeviceToHost, st));
    }
    if (o.stats_out) {
        unsigned long long c[C_COUNT];
        PDX_TRY(cudaMemcpyAsync(c, kc, sizeof c, cudaMemcpyDeviceToHost, st));
        PDX_TRY(cudaStreamSynchronize(st));
        pdx_search_stats *so = o.stats_out;
        std::memset(so, 0, sizeof *so);
        so->values_visited = c[C_VALUES];
        so->vectors_scanned = c[C_SCANNED];
        so->vectors_pruned = c[C_PRUNED];
        so->prune_phase_blocks = c[C_PRUNE_BLOCKS];
        so->candidates = c[C_CANDIDATES];
        so->work_items = c[C_ITEMS];
        so->start_values = c[C_START];
        so->dense_fallbacks = c[C_DENSE_FALLBACK];
        so->bytes_logical = c[C_VALUES] * elem_size(ix->storage) + c[C_START] * 4ull +
                            (ix->storage == PDX_F32 ? 0ull : c[C_CANDIDATES] * (uint64_t)d * 4ull);
        if (ph) ph->fill(so);
    }
    if (!o_dev) PDX_TRY(cudaStreamSynchronize(st));
    return PDX_OK;
}
