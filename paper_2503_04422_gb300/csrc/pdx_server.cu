// Batched serving over many collections: a CUDA-graph-launched exact search
// per (collection, batch bucket) with autotuned launch parameters.
//
// A server owns one device workspace sized for its largest plan, an input and
// an output staging buffer, a private stream, and lazily built entries for
// each (collection, bucket) pair. Buckets are powers of two: a batch of nq
// queries runs in the smallest bucket B >= nq, and rows nq..B-1 of the input
// buffer hold earlier (valid) queries whose results are ignored. On first use
// of an entry the tuner times candidate launch shapes on the caller's batch.
// The shapes are the resident CTAs per SM, the first fetch step and the size
// of a work item in 64-vector blocks. Every candidate gives the same exact
// result. The entry then captures
// the search into a CUDA graph, and later batches replay it after one copy-in.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "pdx_internal.cuh"

namespace pdx {

struct ServerEntry {
    bool ready = false;
    pdx_search_opts opts;
    SearchPlan pl;
    ExactPlan ep;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;  // kernel nodes of the graph: each replay launches them all
    float tuned_ms = 0.f;
};

struct TuneRecord {
    uint32_t ctas, first_step, blocks_per_item;
    float ms;
};

}  // namespace pdx

struct pdx_server {
    std::vector<const pdx_index *> ix;
    pdx_server_opts o;
    int max_bucket_log2 = 0;
    int max_d = 0;
    int sms = 1;
    cudaStream_t st = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    unsigned char *work = nullptr;
    size_t work_bytes = 0;
    float *qbuf = nullptr;
    float *obuf_d = nullptr;
    int64_t *obuf_i = nullptr;
    std::vector<std::vector<pdx::ServerEntry>> entries;  // [collection][bucket]
    std::map<std::string, pdx::TuneRecord> cache;
    std::mutex mu;
    uint64_t graph_launches = 0, direct_launches = 0, tunings = 0;
};

namespace pdx {

static std::string cache_key(const pdx_index *ix, int64_t bucket, int k) {
    char buf[160];
    snprintf(buf, sizeof buf, "n=%lld,d=%d,parts=%d,storage=%d,metric=%d,k=%d,batch=%lld", (long long)ix->n, ix->d,
             ix->nparts, (int)ix->storage, (int)ix->metric, k, (long long)bucket);
    return buf;
}

// Tuner cache file: one JSON object whose keys are cache_key() strings and
// whose values are {"ctas":..,"first_step":..,"blocks_per_item":..,"ms":..}.
static void load_cache(pdx_server *s) {
    if (!s->o.tune_cache) return;
    FILE *f = fopen(s->o.tune_cache, "r");
    if (!f) return;
    std::string txt;
    char buf[4096];
    size_t r;
    while ((r = fread(buf, 1, sizeof buf, f)) > 0) txt.append(buf, r);
    fclose(f);
    size_t pos = 0;
    while ((pos = txt.find('"', pos)) != std::string::npos) {
        size_t e = txt.find('"', pos + 1);
        if (e == std::string::npos) break;
        std::string key = txt.substr(pos + 1, e - pos - 1);
        size_t ob = txt.find('{', e), cb = txt.find('}', e);
        if (ob == std::string::npos || cb == std::string::npos || ob > cb) break;
        std::string body = txt.substr(ob, cb - ob + 1);
        TuneRecord t{};
        unsigned a = 0, b = 0, c = 0;
        float ms = 0.f;
        if (sscanf(body.c_str(), "{\"ctas\": %u, \"first_step\": %u, \"blocks_per_item\": %u, \"ms\": %f}", &a,
                   &b, &c, &ms) == 4) {
            t.ctas = a;
            t.first_step = b;
            t.blocks_per_item = c;
            t.ms = ms;
            s->cache[key] = t;
        }
        pos = cb + 1;
    }
}

static void save_cache(pdx_server *s) {
    if (!s->o.tune_cache) return;
    std::string tmp = std::string(s->o.tune_cache) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n");
    size_t i = 0;
    for (auto &kv : s->cache) {
        fprintf(f, "  \"%s\": {\"ctas\": %u, \"first_step\": %u, \"blocks_per_item\": %u, \"ms\": %.4f}%s\n",
                kv.first.c_str(), kv.second.ctas, kv.second.first_step, kv.second.blocks_per_item, kv.second.ms,
                ++i < s->cache.size() ? "," : "");
    }
    fprintf(f, "}\n");
    fclose(f);
    std::rename(tmp.c_str(), s->o.tune_cache);
}

// Work-item sizes the tuner tries: the automatic one and its half and double.
static std::vector<uint32_t> item_sizes(const pdx_index *ix, int64_t B, int k, const pdx_search_opts &o,
                                        const SearchPlan &pl, int sms) {
    pdx_search_opts a = o;
    a.blocks_per_item = 0;
    ExactPlan ep;
    std::vector<uint32_t> out;
    if (exact_plan(ix, B, k, a, pl, sms, &ep) != PDX_OK || ep.dense || ep.layout) return {o.blocks_per_item};
    for (int b : {ep.bpi, std::max(1, ep.bpi / 2), ep.bpi * 2})
        if (std::find(out.begin(), out.end(), (uint32_t)b) == out.end()) out.push_back((uint32_t)b);
    return out;
}

// A candidate is tried only if its plan fits the server's workspace.
static bool plan_fits(pdx_server *s, const pdx_index *ix, int64_t B, const pdx_search_opts &o, const SearchPlan &pl,
                      uint32_t bpi) {
    pdx_search_opts c = o;
    c.blocks_per_item = bpi;
    ExactPlan ep;
    return exact_plan(ix, B, s->o.k, c, pl, s->sms, &ep) == PDX_OK && ep.bytes <= s->work_bytes;
}

static int bucket_of(int64_t nq) {
    int b = 0;
    while (((int64_t)1 << b) < nq) ++b;
    return b;
}

// Times one candidate on the staged batch (after one untimed run).
static pdx_status time_candidate(pdx_server *s, const pdx_index *ix, int64_t B, const pdx_search_opts &o, float *ms) {
    SearchPlan pl;
    pdx_status r = plan_metric(ix, o.pruner, &pl, "pdx_server_search");
    if (r != PDX_OK) return r;
    ExactPlan ep;
    r = exact_plan(ix, B, s->o.k, o, pl, s->sms, &ep);
    if (r != PDX_OK) return r;
    if (ep.bytes > s->work_bytes) {
        *ms = 1e30f;
        return PDX_OK;
    }
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return PDX_ERR_CUDA;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return PDX_ERR_CUDA;
    }
    r = exact_run(ix, s->qbuf, B, s->o.k, o, pl, ep, s->work, s->obuf_d, s->obuf_i, nullptr, s->sms, s->st);
    if (r == PDX_OK && cudaEventRecord(a, s->st) != cudaSuccess) r = PDX_ERR_CUDA;
    if (r == PDX_OK) r = exact_run(ix, s->qbuf, B, s->o.k, o, pl, ep, s->work, s->obuf_d, s->obuf_i, nullptr, s->sms, s->st);
    if (r == PDX_OK && cudaEventRecord(b, s->st) != cudaSuccess) r = PDX_ERR_CUDA;
    if (r == PDX_OK && cudaEventSynchronize(b) != cudaSuccess) r = PDX_ERR_CUDA;
    if (r == PDX_OK) cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return r;
}

static pdx_status prepare_entry(pdx_server *s, int c, int bk) {
    ServerEntry &E = s->entries[c][bk];
    const pdx_index *ix = s->ix[c];
    const int64_t B = (int64_t)1 << bk;
    pdx_search_opts o = s->o.search;
    // resolve the automatic choices the same way a search would
    pdx_search_opts tmp;
    SearchPlan pl;
    pdx_status r = exact_check(ix, s->qbuf, B, s->o.k, &o, s->obuf_d, s->obuf_i, &tmp, &pl, "pdx_server_search");
    if (r != PDX_OK) return r;
    o = tmp;
    if (s->o.autotune) {
        const std::string key = cache_key(ix, B, s->o.k);
        auto it = s->cache.find(key);
        if (it != s->cache.end()) {
            o.ctas_per_sm = it->second.ctas;
            o.first_step = it->second.first_step;
            o.blocks_per_item = it->second.blocks_per_item;
            E.tuned_ms = it->second.ms;
        } else {
            // candidates: resident CTAs per SM x first fetch step (the first
            // prune-check interval) x work-item size in 64-vector blocks (the
            // automatic size, half of it, twice it), each within the workspace
            float best = 1e30f;
            TuneRecord bt{o.ctas_per_sm, o.first_step, o.blocks_per_item, 0.f};
            const uint32_t ctas[] = {3, 4};
            // a pruner with norms stored for one schedule keeps its first step
            const bool fixed_step = o.pruner == PDX_PRUNE_CS_IP;
            const std::vector<uint32_t> steps =
                fixed_step ? std::vector<uint32_t>{o.first_step} : std::vector<uint32_t>{4u, 8u};
            std::vector<uint32_t> bpis;
            for (uint32_t b : item_sizes(ix, B, s->o.k, o, pl, s->sms))
                if (plan_fits(s, ix, B, o, pl, b)) bpis.push_back(b);
            for (uint32_t ct : ctas)
                for (uint32_t fs : steps)
                    for (uint32_t bp : bpis) {
                        pdx_search_opts c2 = o;
                        c2.ctas_per_sm = ct;
                        c2.first_step = fs;
                        c2.blocks_per_item = bp;
                        float ms = 0.f;
                        r = time_candidate(s, ix, B, c2, &ms);
                        if (r != PDX_OK) return r;
                        if (ms < best) {
                            best = ms;
                            bt = TuneRecord{ct, fs, bp, ms};
                        }
                    }
            o.ctas_per_sm = bt.ctas;
            o.first_step = bt.first_step;
            o.blocks_per_item = bt.blocks_per_item;
            E.tuned_ms = best;
            s->cache[key] = bt;
            s->tunings += 1;
            save_cache(s);
        }
    }
    E.opts = o;
    E.pl = pl;
    r = exact_plan(ix, B, s->o.k, o, pl, s->sms, &E.ep);
    if (r != PDX_OK) return r;
    if (E.ep.bytes > s->work_bytes) {
        set_error("pdx_server_search: internal error: plan needs %zu bytes, workspace has %zu", E.ep.bytes,
                  s->work_bytes);
        return PDX_ERR_CUDA;
    }
    if (s->o.use_graphs) {
        // the scan's launch attributes are set outside capture by one direct run
        r = exact_run(ix, s->qbuf, B, s->o.k, o, pl, E.ep, s->work, s->obuf_d, s->obuf_i, nullptr, s->sms, s->st);
        if (r != PDX_OK) return r;
        cudaError_t e = cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_status_ext(e, "cudaStreamBeginCapture");
        // captured launches run only when the graph is replayed, and are
        // counted then
        const uint64_t before = pdx_kernel_launches();
        r = exact_run(ix, s->qbuf, B, s->o.k, o, pl, E.ep, s->work, s->obuf_d, s->obuf_i, nullptr, s->sms, s->st);
        count_launches(-(int)(pdx_kernel_launches() - before));
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(s->st, &g);
        if (r != PDX_OK) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        if (e != cudaSuccess) return cuda_status_ext(e, "cudaStreamEndCapture");
        E.graph = g;
        size_t nn = 0;
        e = cudaGraphGetNodes(g, nullptr, &nn);
        if (e != cudaSuccess) return cuda_status_ext(e, "cudaGraphGetNodes");
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn > 0) {
            e = cudaGraphGetNodes(g, nodes.data(), &nn);
            if (e != cudaSuccess) return cuda_status_ext(e, "cudaGraphGetNodes");
        }
        E.kernels = 0;
        for (cudaGraphNode_t n : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(n, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++E.kernels;
        }
        e = cudaGraphInstantiate(&E.exec, g, 0);
        if (e != cudaSuccess) return cuda_status_ext(e, "cudaGraphInstantiate");
    }
    E.ready = true;
    return PDX_OK;
}

}  // namespace pdx

using namespace pdx;

extern "C" void pdx_default_server_opts(pdx_server_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->struct_size = sizeof *o;
    o->k = 10;
    o->max_batch = 4096;
    o->use_graphs = 1;
    o->autotune = 1;
    o->tune_cache = nullptr;
    pdx_default_search_opts(&o->search);
}

extern "C" void pdx_server_free(pdx_server *s) {
    if (!s) return;
    for (auto &row : s->entries)
        for (auto &E : row) {
            if (E.exec) cudaGraphExecDestroy(E.exec);
            if (E.graph) cudaGraphDestroy(E.graph);
        }
    if (s->work) cudaFree(s->work);
    if (s->qbuf) cudaFree(s->qbuf);
    if (s->obuf_d) cudaFree(s->obuf_d);
    if (s->obuf_i) cudaFree(s->obuf_i);
    if (s->ev_in) cudaEventDestroy(s->ev_in);
    if (s->ev_out) cudaEventDestroy(s->ev_out);
    if (s->st) cudaStreamDestroy(s->st);
    delete s;
}

extern "C" pdx_status pdx_server_create(const pdx_index *const *indexes, int32_t count, const pdx_server_opts *opts,
                                        pdx_server **out) {
    if (out) *out = nullptr;
    if (!indexes || count < 1 || !out || !opts) {
        set_error("pdx_server_create: NULL argument or count < 1");
        return PDX_ERR_ARG;
    }
    if (opts->struct_size < sizeof(pdx_server_opts) || opts->search.struct_size < sizeof(pdx_search_opts)) {
        set_error("pdx_server_create: struct_size too small");
        return PDX_ERR_ARG;
    }
    if (opts->k < 1 || opts->k > kMaxK || opts->max_batch < 1 || opts->max_batch > (1 << 16)) {
        set_error("pdx_server_create: k=%d max_batch=%d out of range", opts->k, opts->max_batch);
        return PDX_ERR_ARG;
    }
    if (opts->search.pruner != PDX_PRUNE_NONE && opts->search.pruner != PDX_PRUNE_BOND &&
        opts->search.pruner != PDX_PRUNE_CS_IP) {
        set_error("pdx_server_create: a server runs exact searches (pruner NONE, BOND or CS_IP)");
        return PDX_ERR_ARG;
    }
    if (opts->search.tau_init || opts->search.tau_fixed) {
        set_error("pdx_server_create: per-query initial thresholds are a per-call option; a server takes none");
        return PDX_ERR_ARG;
    }
    pdx_server *s = new (std::nothrow) pdx_server();
    if (!s) {
        set_error("host allocation failed");
        return PDX_ERR_OOM;
    }
    s->o = *opts;
    s->max_bucket_log2 = bucket_of(opts->max_batch);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
    if (s->sms < 1) s->sms = 1;
    const int64_t Bmax = (int64_t)1 << s->max_bucket_log2;
    // size the workspace for the largest plan over all collections and the
    // candidate shapes the tuner may try
    for (int c = 0; c < count; ++c) {
        const pdx_index *ix = indexes[c];
        if (!ix || ix->is_ivf) {
            pdx_server_free(s);
            set_error("pdx_server_create: collection %d is NULL or an IVF index", c);
            return PDX_ERR_ARG;
        }
        s->ix.push_back(ix);
        s->max_d = std::max(s->max_d, ix->d);
        pdx_search_opts o;
        SearchPlan pl;
        pdx_search_opts base = opts->search;
        pdx_status r = check_search_args(ix, nullptr, 0, opts->k, &base, nullptr, nullptr, &o, "pdx_server_create");
        if (r == PDX_OK) r = plan_metric(ix, o.pruner, &pl, "pdx_server_create");
        if (r != PDX_OK) {
            pdx_server_free(s);
            return r;
        }
        for (int bk = 0; bk <= s->max_bucket_log2; ++bk) {
            // the automatic plan always fits; the tuner's other item sizes fit
            // when their lists stay within 256 MB more
            const int64_t B = (int64_t)1 << bk;
            ExactPlan ep;
            exact_plan(ix, B, opts->k, o, pl, s->sms, &ep);
            size_t need = ep.bytes;
            if (opts->autotune) {
                for (uint32_t b : item_sizes(ix, B, opts->k, o, pl, s->sms)) {
                    pdx_search_opts c = o;
                    c.blocks_per_item = b;
                    ExactPlan e2;
                    if (exact_plan(ix, B, opts->k, c, pl, s->sms, &e2) == PDX_OK && e2.bytes <= ep.bytes + ((size_t)256 << 20))
                        need = std::max(need, e2.bytes);
                }
            }
            s->work_bytes = std::max(s->work_bytes, need);
        }
    }
    s->entries.assign(count, std::vector<ServerEntry>(s->max_bucket_log2 + 1));
    cudaError_t e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&s->work, s->work_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->qbuf, (size_t)Bmax * s->max_d * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->obuf_d, (size_t)Bmax * opts->k * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->obuf_i, (size_t)Bmax * opts->k * 8);
    if (e == cudaSuccess) e = cudaMemset(s->qbuf, 0, (size_t)Bmax * s->max_d * 4);
    if (e != cudaSuccess) {
        set_error("pdx_server_create: %s", cudaGetErrorString(e));
        pdx_server_free(s);
        return e == cudaErrorMemoryAllocation ? PDX_ERR_OOM : PDX_ERR_CUDA;
    }
    load_cache(s);
    *out = s;
    return PDX_OK;
}

extern "C" pdx_status pdx_server_search(pdx_server *s, int32_t collection, const float *q, int64_t nq,
                                        float *out_dist, int64_t *out_idx, void *stream) {
    const char *fn = "pdx_server_search";
    if (!s || (nq > 0 && (!q || !out_dist || !out_idx))) {
        set_error("%s: NULL argument", fn);
        return PDX_ERR_ARG;
    }
    if (collection < 0 || collection >= (int)s->ix.size() || nq < 0 || nq > s->o.max_batch) {
        set_error("%s: collection %d or batch %lld out of range (max_batch %d)", fn, collection, (long long)nq,
                  s->o.max_batch);
        return PDX_ERR_ARG;
    }
    if (nq == 0) return PDX_OK;
    std::lock_guard<std::mutex> lk(s->mu);
    const pdx_index *ix = s->ix[collection];
    const int d = ix->d, k = s->o.k;
    const int bk = bucket_of(nq);
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    cudaPointerAttributes qa, oa;
    bool q_dev = cudaPointerGetAttributes(&qa, q) == cudaSuccess &&
                 (qa.type == cudaMemoryTypeDevice || qa.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    bool o_dev = cudaPointerGetAttributes(&oa, out_dist) == cudaSuccess &&
                 (oa.type == cudaMemoryTypeDevice || oa.type == cudaMemoryTypeManaged);
    cudaGetLastError();
#define SRV_TRY(call)                                                                                     \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) {                                                                          \
            set_error("%s: %s failed: %s", fn, #call, cudaGetErrorString(e_));                            \
            return e_ == cudaErrorMemoryAllocation ? PDX_ERR_OOM : PDX_ERR_CUDA;                          \
        }                                                                                                 \
    } while (0)
    // order the private stream after the caller's work, stage the batch
    SRV_TRY(cudaEventRecord(s->ev_in, caller));
    SRV_TRY(cudaStreamWaitEvent(s->st, s->ev_in, 0));
    SRV_TRY(cudaMemcpyAsync(s->qbuf, q, (size_t)nq * d * 4, q_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            s->st));
    ServerEntry &E = s->entries[collection][bk];
    if (!E.ready) {
        pdx_status r = prepare_entry(s, collection, bk);
        if (r != PDX_OK) return r;
    }
    if (E.exec) {
        SRV_TRY(cudaGraphLaunch(E.exec, s->st));
        count_launches(E.kernels);
        s->graph_launches += 1;
    } else {
        pdx_status r = exact_run(ix, s->qbuf, (int64_t)1 << bk, k, E.opts, E.pl, E.ep, s->work, s->obuf_d, s->obuf_i,
                                 nullptr, s->sms, s->st);
        if (r != PDX_OK) return r;
        s->direct_launches += 1;
    }
    const cudaMemcpyKind dk = o_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    SRV_TRY(cudaMemcpyAsync(out_dist, s->obuf_d, (size_t)nq * k * 4, dk, s->st));
    SRV_TRY(cudaMemcpyAsync(out_idx, s->obuf_i, (size_t)nq * k * 8, dk, s->st));
    SRV_TRY(cudaEventRecord(s->ev_out, s->st));
    SRV_TRY(cudaStreamWaitEvent(caller, s->ev_out, 0));
    if (!o_dev) SRV_TRY(cudaStreamSynchronize(s->st));
#undef SRV_TRY
    return PDX_OK;
}

extern "C" pdx_status pdx_server_info(const pdx_server *s, pdx_server_info_t *info) {
    if (!s || !info) {
        set_error("pdx_server_info: NULL argument");
        return PDX_ERR_ARG;
    }
    info->collections = (int32_t)s->ix.size();
    info->max_bucket = 1 << s->max_bucket_log2;
    info->workspace_bytes = s->work_bytes;
    info->graph_launches = s->graph_launches;
    info->direct_launches = s->direct_launches;
    info->tunings = s->tunings;
    int ready = 0;
    for (auto &row : s->entries)
        for (auto &E : row) ready += E.ready ? 1 : 0;
    info->entries_ready = ready;
    return PDX_OK;
}
