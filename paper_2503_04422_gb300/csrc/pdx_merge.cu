// Merge of per-shard top-k lists: the exchange step of a collection sharded
// across GPUs or processes. Each shard searches its part of the collection
// (ids already made global), the lists are gathered, and this merge keeps the
// k best (distance, id) pairs per query in the order the searches use: L2/L1
// ascending, IP descending, ties to the lower id, padding (id -1) last.
// Host pointers are merged on the calling thread, so the step also runs on a
// host without a GPU; device pointers are merged by one kernel on `stream`.
#include <cstring>
#include <limits>
#include <vector>

#include "pdx_internal.cuh"

namespace pdx {
namespace {

constexpr float kInf = std::numeric_limits<float>::infinity();

// (rank value, id) with padding as +inf: smaller is better.
struct MergeKey {
    float v;
    int64_t id;
};

__host__ __device__ inline MergeKey merge_key(float dist, int64_t id, int metric) {
    MergeKey m;
    if (id < 0) {
        m.v = kInf;
        m.id = INT64_MAX;
    } else {
        m.v = metric == PDX_IP ? -dist : dist;
        m.id = id;
    }
    return m;
}

__host__ __device__ inline bool better(const MergeKey &a, const MergeKey &b) {
    return a.v < b.v || (a.v == b.v && a.id < b.id);
}

// Serial k-way merge of one query's nshards sorted rows.
__host__ __device__ inline void merge_row(const float *dist, const int64_t *idx, int32_t nshards, int64_t nq, int32_t k,
                                          int64_t row, int metric, int32_t *head, float *od, int64_t *oi) {
    for (int s = 0; s < nshards; ++s) head[s] = 0;
    for (int r = 0; r < k; ++r) {
        int best = -1;
        MergeKey bk;
        for (int s = 0; s < nshards; ++s) {
            if (head[s] >= k) continue;
            const int64_t at = ((int64_t)s * nq + row) * k + head[s];
            const MergeKey c = merge_key(dist[at], idx[at], metric);
            if (best < 0 || better(c, bk)) {
                best = s;
                bk = c;
            }
        }
        const int64_t at = ((int64_t)best * nq + row) * k + head[best];
        if (idx[at] < 0) {
            od[row * k + r] = metric == PDX_IP ? -kInf : kInf;
            oi[row * k + r] = -1;
        } else {
            od[row * k + r] = dist[at];
            oi[row * k + r] = idx[at];
        }
        head[best] += 1;
    }
}

constexpr int kMaxShards = 64;

__global__ void merge_topk_kernel(const float *dist, const int64_t *idx, int32_t nshards, int64_t nq, int32_t k,
                                  int metric, float *od, int64_t *oi) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= nq) return;
    int32_t head[kMaxShards];
    merge_row(dist, idx, nshards, nq, k, row, metric, head, od, oi);
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace pdx

using namespace pdx;

extern "C" pdx_status pdx_merge_topk(const float *dist, const int64_t *idx, int32_t nshards, int64_t nq, int32_t k,
                                     pdx_metric metric, float *out_dist, int64_t *out_idx, void *stream) {
    if (nshards < 1 || nshards > kMaxShards || nq < 0 || k < 1 || k > kMaxK ||
        (metric != PDX_L2 && metric != PDX_IP && metric != PDX_L1)) {
        set_error("pdx_merge_topk: nshards=%d (1..%d), nq=%lld, k=%d or metric %d out of range", nshards, kMaxShards,
                  (long long)nq, k, (int)metric);
        return PDX_ERR_ARG;
    }
    if (nq == 0) return PDX_OK;
    if (!dist || !idx || !out_dist || !out_idx) {
        set_error("pdx_merge_topk: NULL argument");
        return PDX_ERR_ARG;
    }
    const bool dev[4] = {on_device(dist), on_device(idx), on_device(out_dist), on_device(out_idx)};
    if (dev[0] != dev[1] || dev[0] != dev[2] || dev[0] != dev[3]) {
        set_error("pdx_merge_topk: inputs and outputs must all be host or all be device pointers");
        return PDX_ERR_ARG;
    }
    if (!dev[0]) {
        std::vector<int32_t> head((size_t)nshards);
        for (int64_t r = 0; r < nq; ++r) merge_row(dist, idx, nshards, nq, k, r, metric, head.data(), out_dist, out_idx);
        return PDX_OK;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    merge_topk_kernel<<<(unsigned)((nq + 127) / 128), 128, 0, st>>>(dist, idx, nshards, nq, k, (int)metric, out_dist,
                                                                    out_idx);
    cudaError_t e = counted(cudaGetLastError());
    if (e != cudaSuccess) return cuda_status_ext(e, "merge_topk_kernel");
    return PDX_OK;
}
