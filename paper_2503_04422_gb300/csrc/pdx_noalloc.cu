// pdx_search_exact_noalloc: the exact search with its scratch memory in a
// fixed, statically declared device array instead of the stream-ordered
// allocator. It launches the same kernels as pdx_search_exact.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "pdx_internal.cuh"

namespace pdx {

// Capacity of the static scratch array. Every GPU that loads the library
// holds this much device memory until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kNoAllocMaxDevices = 64;

// Shared by every call of pdx_search_exact_noalloc on a device. Host code
// must not use this symbol as a device address: its name denotes a host-side
// shadow. The device address is looked up once per device with
// cudaGetSymbolAddress (noalloc_scratch below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_dev_ptr[kNoAllocMaxDevices] = {};

// Device address of the static scratch array on the current device. Looked up
// on the first call made with that device current; later calls reuse it.
static pdx_status noalloc_scratch(unsigned char **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error("pdx_search_exact_noalloc: cudaGetDevice failed: %s", cudaGetErrorString(e));
        return PDX_ERR_CUDA;
    }
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("pdx_search_exact_noalloc: device ordinal %d not supported", dev);
        return PDX_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_dev_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("pdx_search_exact_noalloc: cudaGetSymbolAddress of the scratch array failed: %s",
                      cudaGetErrorString(e));
            return PDX_ERR_CUDA;
        }
        g_noalloc_dev_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_noalloc_dev_ptr[dev];
    return PDX_OK;
}

static bool noalloc_is_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static size_t r256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace pdx

using namespace pdx;

extern "C" pdx_status pdx_search_exact_noalloc(const pdx_index *ix, const float *q, int64_t nq, int32_t k,
                                               const pdx_search_opts *opts, float *out_dist, int64_t *out_idx,
                                               void *stream) {
    const char *fn = "pdx_search_exact_noalloc";
    pdx_search_opts o;
    pdx_status s = check_search_args(ix, q, nq, k, opts, out_dist, out_idx, &o, fn);
    if (s != PDX_OK) return s;
    if (ix->is_ivf) {
        set_error("%s: index was built by pdx_ivf_build", fn);
        return PDX_ERR_ARG;
    }
    if (o.pruner != PDX_PRUNE_NONE && o.pruner != PDX_PRUNE_BOND) {
        set_error("%s: only NONE or BOND keep the search exact", fn);
        return PDX_ERR_ARG;
    }
    SearchPlan pl;
    s = plan_metric(ix, o.pruner, &pl, fn);
    if (s != PDX_OK) return s;
    if (nq == 0) return PDX_OK;
    if (!noalloc_is_device(q) || !noalloc_is_device(out_dist) || !noalloc_is_device(out_idx)) {
        set_error("%s: q, out_dist and out_idx must be device memory (this entry point stages nothing)", fn);
        return PDX_ERR_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int d = ix->d;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;

    int max_blk = 0;
    for (int p = 0; p < ix->nparts; ++p) max_blk = std::max(max_blk, ix->h_part_blk[p + 1] - ix->h_part_blk[p]);
    int bpi = (int)o.blocks_per_item;
    if (bpi <= 0) {
        const int64_t target = (int64_t)sms * 64 * 3;
        int64_t pairs = nq * (int64_t)ix->nparts;
        int chunks = (int)std::min<int64_t>(max_blk, std::max<int64_t>(1, (target + pairs - 1) / pairs));
        bpi = (max_blk + chunks - 1) / chunks;
    }
    if (bpi < 1) bpi = 1;
    const int chunks = (max_blk + bpi - 1) / bpi;
    const int nslots = ix->nparts * chunks;
    const bool start = (pl.pruner != PDX_PRUNE_NONE);
    int start_blk = 0;
    if (start) {
        int64_t sv = std::max<int64_t>(o.start_vectors, k);
        start_blk = (int)std::min<int64_t>(ix->nblocks, (sv + kBlock - 1) / kBlock);
    }
    const int64_t Lstart = (int64_t)start_blk * kBlock;

    const OrderPlan op = plan_orders(ix, o, pl.pruner, nq, ix->nparts);
    size_t need = r256((size_t)nq * 4) + r256((size_t)nq * nslots * k * 8) + 3 * r256((size_t)nq * k * 8) +
                  r256(C_COUNT * 8) + r256(8) + r256(op.bytes);
    if (start) need += r256((size_t)nq * Lstart * 8) + r256((size_t)nq * k * 8);
    if (need > kNoAllocScratchBytes) {
        set_error("%s: this search needs %zu bytes of scratch but the static array holds %zu; "
                  "use fewer queries per call or a smaller start_vectors", fn, need, kNoAllocScratchBytes);
        return PDX_ERR_ARG;
    }
    unsigned char *base = nullptr;
    s = noalloc_scratch(&base);
    if (s != PDX_OK) return s;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char *p = base + off;
        off += r256(bytes);
        return p;
    };
    float *tau = reinterpret_cast<float *>(take((size_t)nq * 4));
    uint64_t *cand = reinterpret_cast<uint64_t *>(take((size_t)nq * nslots * k * 8));
    uint64_t *topk = reinterpret_cast<uint64_t *>(take((size_t)nq * k * 8));
    uint64_t *refined = reinterpret_cast<uint64_t *>(take((size_t)nq * k * 8));
    uint64_t *final_keys = reinterpret_cast<uint64_t *>(take((size_t)nq * k * 8));
    unsigned long long *counters = reinterpret_cast<unsigned long long *>(take(C_COUNT * 8));
    int *work = reinterpret_cast<int *>(take(8));
    uint64_t *skeys = start ? reinterpret_cast<uint64_t *>(take((size_t)nq * Lstart * 8)) : nullptr;
    uint64_t *stopk = start ? reinterpret_cast<uint64_t *>(take((size_t)nq * k * 8)) : nullptr;
    uint16_t *qorder = op.rows ? reinterpret_cast<uint16_t *>(take(op.bytes)) : nullptr;

#define NOALLOC_TRY(call)                                                                             \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) {                                                                      \
            set_error("%s: %s failed: %s", fn, #call, cudaGetErrorString(e_));                        \
            return PDX_ERR_CUDA;                                                                      \
        }                                                                                             \
    } while (0)

    // the array keeps the previous call's contents: reset everything that must
    // start from a known value (thresholds, counters, the work counter)
    if (op.rows)
        NOALLOC_TRY(launch_order(q, op.rows, d, op.per_part ? ix->means : ix->cmean, op.per_part, nullptr, op.mode,
                                 std::max(1, (int)o.zone_dims), qorder, st));
    NOALLOC_TRY(launch_fill_u32(reinterpret_cast<uint32_t *>(tau), 0xff800000u, nq, st));
    NOALLOC_TRY(cudaMemsetAsync(counters, 0, C_COUNT * 8, st));
    NOALLOC_TRY(cudaMemsetAsync(work, 0, 8, st));
    unsigned long long *kc = o.stats_device ? reinterpret_cast<unsigned long long *>(o.stats_device) : counters;
    if (start) {
        if (ix->storage == PDX_F32) {
            NOALLOC_TRY(launch_dense_keys(q, nq, ix->data, ix->ids, d, start_blk, pl.metric, skeys, st));
        } else {
            const int32_t rows = (int32_t)std::min<int64_t>(ix->n, Lstart);
            NOALLOC_TRY(launch_fill_u64(skeys, kEmptyKey, nq * Lstart, st));
            NOALLOC_TRY(launch_dense_keys_rows(q, nq, ix->xnary, rows, d, Lstart, skeys, st));
        }
        NOALLOC_TRY(launch_select_k(skeys, nq, Lstart, k, stopk, st));
        NOALLOC_TRY(launch_tau_from_keys(stopk, nq, k, tau, st));
        NOALLOC_TRY(launch_add_u64(kc + C_START, (unsigned long long)nq * Lstart * d, st));
    }
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
    p.q = q;
    p.nq = nq;
    p.means = ix->means;
    p.nslots = nslots;
    p.chunks_per_part = chunks;
    p.blocks_per_item = bpi;
    p.k = k;
    p.tau = tau;
    p.cand = cand;
    p.counters = kc;
    p.work_counter = work;
    p.nitems = nq * (int64_t)nslots;
    p.first_step = (int)o.first_step;
    p.sel_count = std::min(kMaxSurv, (int)std::ceil(o.selection_threshold * kBlock) - 1);
    if (p.sel_count < 0) p.sel_count = 0;
    p.zone_dims = (int)o.zone_dims;
    p.order = (int)o.order;
    p.ctas_per_sm = (int)o.ctas_per_sm;
    p.gamma = (float)d * 1.1920929e-7f;
    p.eps0 = o.eps0;
    p.bsa_m = o.bsa_m;
    p.qorder = qorder;
    p.qorder_per_part = op.per_part;
    if (o.scan_event_start) NOALLOC_TRY(cudaEventRecord(static_cast<cudaEvent_t>(o.scan_event_start), st));
    NOALLOC_TRY(launch_scan(pl.pruner, pl.metric, p, sms, st));
    if (o.scan_event_stop) NOALLOC_TRY(cudaEventRecord(static_cast<cudaEvent_t>(o.scan_event_stop), st));
    NOALLOC_TRY(launch_select_k(cand, nq, (int64_t)nslots * k, k, topk, st));
    if (ix->storage == PDX_F32)
        NOALLOC_TRY(launch_refine(topk, nq, k, q, d, ix->data, ix->slot_of, ix->metric, refined, st));
    else
        NOALLOC_TRY(launch_refine_rows(topk, nq, k, q, d, ix->xnary, ix->metric, refined, st));
    NOALLOC_TRY(launch_select_k(refined, nq, k, k, final_keys, st));
    NOALLOC_TRY(launch_write_out(final_keys, nq, k, pl.out_mode, q, d, out_dist, out_idx, st));
    if (o.stats_out) {
        unsigned long long c[C_COUNT];
        NOALLOC_TRY(cudaMemcpyAsync(c, kc, sizeof c, cudaMemcpyDeviceToHost, st));
        NOALLOC_TRY(cudaStreamSynchronize(st));
        pdx_search_stats *so = o.stats_out;
        std::memset(so, 0, sizeof *so);
        so->values_visited = c[C_VALUES];
        so->vectors_scanned = c[C_SCANNED];
        so->vectors_pruned = c[C_PRUNED];
        so->prune_phase_blocks = c[C_PRUNE_BLOCKS];
        so->candidates = c[C_CANDIDATES];
        so->work_items = c[C_ITEMS];
        so->start_values = c[C_START];
        so->bytes_logical = c[C_VALUES] * (ix->storage == PDX_F32 ? 4ull : (ix->storage == PDX_BF16 ? 2ull : 1ull)) +
                            c[C_START] * 4ull + (ix->storage == PDX_F32 ? 0ull : c[C_CANDIDATES] * (uint64_t)d * 4ull);
    }
#undef NOALLOC_TRY
    return PDX_OK;
}
