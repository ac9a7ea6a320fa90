// Linear-scan kernels over four storage layouts (Sec. 3, Fig. 3; the distance
// kernel study of Sec. 6.2 / Table 3; N-ary + gather in Sec. 7; DSM in
// Sec. 7 "PDX vs DSM"). They answer the same exact k-NN as the PDX scan
// without a pruner, so the layouts can be compared on one workload:
//
//   PDX     blocks of 64 vectors stored dimension-major (element (t, j) of
//           block b at (b*D + j)*64 + t): lanes own vectors, a 16-byte load
//           covers 4 vectors of one dimension, no reduction across lanes.
//   DSM     the whole collection dimension-major (element (i, j) at
//           j*n_pad + i): the same lane mapping, but consecutive dimensions
//           of a block are n_pad*4 bytes apart instead of 256.
//   N-ary   row-major vectors (x[i*D + j]), the horizontal layout: a warp
//           takes four vectors at a time, lanes take 16-byte pieces of their
//           rows and each vector's partial sums are reduced across the warp
//           at its end (the reduction the PDX kernel avoids).
//   GATHER  row-major vectors transposed on the fly: a warp stages a tile of
//           64 vectors x 32 dimensions from the rows into shared memory and
//           runs the PDX kernel on the tile.
//
// Work item: (query, chunk of kChunkBlocks 64-vector blocks); one warp per
// item, pulled from a global counter. Each item leaves its k best (distance,
// id) keys; the host merges them like the PDX scan's per-item lists.
#include <algorithm>
#include <cstring>

#include "pdx_internal.cuh"

namespace pdx {

namespace {

constexpr int kChunkBlocks = 16;   // 1024 vectors per work item
constexpr int kLayoutWarps = 8;
constexpr int kTilePitch = 65;     // GATHER tile row pitch (floats): conflict-free transposed stores

struct LayoutParams {
    int layout;
    const float *x;            // PDX blocks, DSM columns or rows (by layout)
    const int32_t *ids;        // PDX: slot -> id (-1 padding)
    int64_t n;
    int64_t n_pad;             // DSM column length (multiple of 64)
    int64_t nblk;              // 64-vector blocks scanned (PDX: the index's blocks, whose
                               // partitions each end in a padded block; else ceil(n/64))
    int32_t d;
    const float *q;
    int64_t nq;
    int32_t k;
    int64_t nchunks;
    uint64_t *cand;            // [nq][nchunks][k]
    int *work_counter;
    int64_t nitems;
};

// Insert key into the warp's ascending list (capacity k, count cnt). Warp-uniform.
__device__ __forceinline__ void list_insert(uint64_t *list, int &cnt, int k, uint64_t key, int lane) {
    if (cnt == k && key >= list[k - 1]) return;
    int pos = 0;
    for (int base = 0; base < cnt; base += 32) {
        const int i = base + lane;
        pos += __popc(__ballot_sync(kFull, i < cnt && list[i] < key));
    }
    const int top = cnt < k ? cnt : k - 1;
    for (int base = (top >> 5) << 5; base >= 0; base -= 32) {
        const int i = base + lane;
        const bool mv = i > pos && i <= top;
        const uint64_t v = mv ? list[i - 1] : 0ull;
        __syncwarp();
        if (mv) list[i] = v;
        __syncwarp();
        if (base <= pos) break;
    }
    if (lane == 0) list[pos] = key;
    __syncwarp();
    if (cnt < k) ++cnt;
}

// Offer the 4 distances a lane holds (vectors 4*sl+c of a 64-vector group,
// valid if id >= 0) to the warp's list; lanes h == 1 hold copies and offer none.
__device__ __forceinline__ void offer4(uint64_t *list, int &cnt, int k, const float (&dist)[4], const int (&id)[4],
                                       bool mine, int lane) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float kth = (cnt == k) ? key_dist(list[k - 1]) : __int_as_float(0x7f800000);
        const bool cand = mine && id[c] >= 0 && dist[c] <= kth;
        unsigned m = __ballot_sync(kFull, cand);
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1u;
            const float dd = __shfl_sync(kFull, dist[c], src);
            const int ii = __shfl_sync(kFull, id[c], src);
            list_insert(list, cnt, k, make_key(dd, ii), lane);
        }
    }
}

template <int MET, int LAYOUT>
__global__ void __launch_bounds__(kLayoutWarps * 32) layout_scan_kernel(LayoutParams a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int D = a.d, k = a.k;
    const int h = lane >> 4, sl = lane & 15;
    // per warp: the list (k keys), the query (D floats), and the GATHER tile
    const size_t list_bytes = ((size_t)k * 8 + 15) & ~size_t(15);
    const size_t q_bytes = ((size_t)D * 4 + 15) & ~size_t(15);
    const size_t tile_bytes = (LAYOUT == PDX_LAYOUT_NARY_GATHER) ? (size_t)32 * kTilePitch * 4 : 0;
    unsigned char *wbase = smem + (size_t)warp * (list_bytes + q_bytes + tile_bytes);
    uint64_t *list = reinterpret_cast<uint64_t *>(wbase);
    float *qs = reinterpret_cast<float *>(wbase + list_bytes);
    float *tile = reinterpret_cast<float *>(wbase + list_bytes + q_bytes);
    const int64_t nblk = a.nblk;

    while (true) {
        unsigned long long wi = 0;
        if (lane == 0) wi = atomicAdd(reinterpret_cast<unsigned long long *>(a.work_counter), 1ull);
        wi = __shfl_sync(kFull, wi, 0);
        if ((int64_t)wi >= a.nitems) break;
        const int64_t chunk = (int64_t)(wi / (unsigned long long)a.nq);
        const int64_t qi = (int64_t)(wi % (unsigned long long)a.nq);
        const float *qrow = a.q + qi * D;
        for (int j = lane; j < D; j += 32) qs[j] = qrow[j];
        __syncwarp();
        int cnt = 0;
        const int64_t b0 = chunk * kChunkBlocks, b1 = min(nblk, b0 + kChunkBlocks);
        for (int64_t b = b0; b < b1; ++b) {
            if (LAYOUT == PDX_LAYOUT_NARY) {
                // four vectors at a time: lanes take 16-byte pieces of their
                // rows (four rows' loads in flight), then each vector's partial
                // sums are reduced across the warp
                const int n4 = D >> 2;
                const int64_t v0 = b * kBlock;
                const int vend = (int)min((int64_t)kBlock, a.n - v0);
                for (int t = 0; t < vend; t += 4) {
                    float acc[4] = {0.f, 0.f, 0.f, 0.f};
                    const float4 *row[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        row[r] = reinterpret_cast<const float4 *>(a.x + (v0 + min(t + r, vend - 1)) * D);
                    for (int i = lane; i < n4; i += 32) {
                        float4 xv[4];
#pragma unroll
                        for (int r = 0; r < 4; ++r) xv[r] = __ldg(row[r] + i);
                        const float4 qv = *reinterpret_cast<const float4 *>(qs + 4 * i);
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            acc[r] = term<MET>(qv.x, xv[r].x, acc[r]);
                            acc[r] = term<MET>(qv.y, xv[r].y, acc[r]);
                            acc[r] = term<MET>(qv.z, xv[r].z, acc[r]);
                            acc[r] = term<MET>(qv.w, xv[r].w, acc[r]);
                        }
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        if (t + r >= vend) break;
                        const float dist = rank_dist<MET>(warp_sum(acc[r]));
                        const float kth = (cnt == k) ? key_dist(list[k - 1]) : __int_as_float(0x7f800000);
                        if (dist <= kth) list_insert(list, cnt, k, make_key(dist, (int)(v0 + t + r)), lane);
                    }
                }
                continue;
            }
            // PDX, DSM, GATHER: lane (h, sl) accumulates vectors 4*sl..+3 over
            // the dimensions of parity h; the halves are added at the end
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            if (LAYOUT == PDX_LAYOUT_PDX_KERNEL || LAYOUT == PDX_LAYOUT_DSM) {
                const float *base = (LAYOUT == PDX_LAYOUT_PDX_KERNEL) ? a.x + (size_t)b * D * kBlock : a.x + (size_t)b * kBlock;
                const int64_t ld = (LAYOUT == PDX_LAYOUT_PDX_KERNEL) ? kBlock : a.n_pad;
                int j = h;
                for (; j + 6 < D; j += 8) {  // 4 loads in flight per lane
                    float4 xv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        xv[u] = __ldg(reinterpret_cast<const float4 *>(base + (int64_t)(j + 2 * u) * ld + 4 * sl));
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float qv = qs[j + 2 * u];
                        acc.x = term<MET>(qv, xv[u].x, acc.x);
                        acc.y = term<MET>(qv, xv[u].y, acc.y);
                        acc.z = term<MET>(qv, xv[u].z, acc.z);
                        acc.w = term<MET>(qv, xv[u].w, acc.w);
                    }
                }
                for (; j < D; j += 2) {
                    const float4 xv = __ldg(reinterpret_cast<const float4 *>(base + (int64_t)j * ld + 4 * sl));
                    const float qv = qs[j];
                    acc.x = term<MET>(qv, xv.x, acc.x);
                    acc.y = term<MET>(qv, xv.y, acc.y);
                    acc.z = term<MET>(qv, xv.z, acc.z);
                    acc.w = term<MET>(qv, xv.w, acc.w);
                }
            } else {
                // GATHER: 64 rows x 32 dimensions per tile, read row by row
                // (8 lanes x 16 bytes per row) and stored transposed
                const int64_t v0 = b * kBlock;
                const int nv = (int)min((int64_t)kBlock, a.n - v0);
                for (int t0 = 0; t0 < D; t0 += 32) {
                    const int tw = min(32, D - t0);
#pragma unroll 4
                    for (int u = 0; u < 16; ++u) {
                        const int e = (u * 32 + lane) * 4;  // element of the 64 x 32 tile
                        const int r = e >> 5, c = e & 31;
                        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (r < nv && c < tw) v = __ldg(reinterpret_cast<const float4 *>(a.x + (v0 + r) * D + t0 + c));
                        tile[(c + 0) * kTilePitch + r] = v.x;
                        tile[(c + 1) * kTilePitch + r] = v.y;
                        tile[(c + 2) * kTilePitch + r] = v.z;
                        tile[(c + 3) * kTilePitch + r] = v.w;
                    }
                    __syncwarp();
                    for (int j = h; j < tw; j += 2) {
                        const float *trow = tile + j * kTilePitch + 4 * sl;
                        const float qv = qs[t0 + j];
                        acc.x = term<MET>(qv, trow[0], acc.x);
                        acc.y = term<MET>(qv, trow[1], acc.y);
                        acc.z = term<MET>(qv, trow[2], acc.z);
                        acc.w = term<MET>(qv, trow[3], acc.w);
                    }
                    __syncwarp();
                }
            }
            float dist[4];
            dist[0] = rank_dist<MET>(acc.x + __shfl_xor_sync(kFull, acc.x, 16));
            dist[1] = rank_dist<MET>(acc.y + __shfl_xor_sync(kFull, acc.y, 16));
            dist[2] = rank_dist<MET>(acc.z + __shfl_xor_sync(kFull, acc.z, 16));
            dist[3] = rank_dist<MET>(acc.w + __shfl_xor_sync(kFull, acc.w, 16));
            int id[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t slot = b * kBlock + 4 * sl + c;
                if (LAYOUT == PDX_LAYOUT_PDX_KERNEL)
                    id[c] = a.ids[slot];
                else
                    id[c] = slot < a.n ? (int)slot : -1;
            }
            offer4(list, cnt, k, dist, id, h == 0, lane);
        }
        uint64_t *out = a.cand + ((size_t)qi * a.nchunks + chunk) * k;
        for (int i = lane; i < k; i += 32) out[i] = (i < cnt) ? list[i] : kEmptyKey;
        __syncwarp();
    }
}

template <int LAYOUT>
cudaError_t launch_layout_t(int metric, const LayoutParams &p, size_t smem, int grid, cudaStream_t st) {
    cudaError_t e;
    switch (metric) {
    case MT_IP:
        e = raise_smem_limit(layout_scan_kernel<MT_IP, LAYOUT>, smem);
        if (e != cudaSuccess) return e;
        layout_scan_kernel<MT_IP, LAYOUT><<<grid, kLayoutWarps * 32, smem, st>>>(p);
        break;
    case MT_L1:
        e = raise_smem_limit(layout_scan_kernel<MT_L1, LAYOUT>, smem);
        if (e != cudaSuccess) return e;
        layout_scan_kernel<MT_L1, LAYOUT><<<grid, kLayoutWarps * 32, smem, st>>>(p);
        break;
    default:
        e = raise_smem_limit(layout_scan_kernel<MT_L2, LAYOUT>, smem);
        if (e != cudaSuccess) return e;
        layout_scan_kernel<MT_L2, LAYOUT><<<grid, kLayoutWarps * 32, smem, st>>>(p);
    }
    return counted(cudaGetLastError());
}

size_t warp_bytes(int layout, int d, int k) {
    return (((size_t)k * 8 + 15) & ~size_t(15)) + (((size_t)d * 4 + 15) & ~size_t(15)) +
           (layout == PDX_LAYOUT_NARY_GATHER ? (size_t)32 * kTilePitch * 4 : 0);
}

__global__ void dsm_transpose_kernel(const float *__restrict__ x, int64_t n, int32_t d, int64_t n_pad,
                                     float *__restrict__ out) {
    // 32 x 32 tiles through shared memory: reads along rows, writes along columns
    __shared__ float t[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32;
    const int j0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = i0 + r;
        const int j = j0 + threadIdx.x;
        t[r][threadIdx.x] = (i < n && j < d) ? x[i * d + j] : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = j0 + r;
        const int64_t i = i0 + threadIdx.x;
        if (j < d && i < n_pad) out[(int64_t)j * n_pad + i] = t[threadIdx.x][r];
    }
}

}  // namespace

cudaError_t launch_dsm_transpose(const float *x, int64_t n, int32_t d, int64_t n_pad, float *out, cudaStream_t st) {
    dim3 grid((unsigned)((n_pad + 31) / 32), (unsigned)((d + 31) / 32));
    dsm_transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(x, n, d, n_pad, out);
    return counted(cudaGetLastError());
}

bool layout_supported(const pdx_index *ix, int layout, int32_t k, const char **why) {
    const char *w = nullptr;
    if (ix->is_ivf) w = "layout scans serve exact indexes";
    else if (ix->storage != PDX_F32) w = "layout scans read FP32 vectors";
    else if (k > 256) w = "layout scans keep at most 256 results per query";
    else if (layout == PDX_LAYOUT_PDX_KERNEL && !ix->data) w = "the index keeps no FP32 PDX blocks";
    else if ((layout == PDX_LAYOUT_NARY || layout == PDX_LAYOUT_NARY_GATHER) && !ix->xnary)
        w = "the index keeps no row-major vectors (build with keep_rows)";
    else if ((layout == PDX_LAYOUT_NARY || layout == PDX_LAYOUT_NARY_GATHER) && ix->d % 4 != 0)
        w = "N-ary layout scans need d to be a multiple of 4";
    else if (layout == PDX_LAYOUT_DSM && !ix->dsm) w = "the index keeps no DSM columns (build with keep_dsm)";
    if (why) *why = w;
    return w == nullptr;
}

// 64-vector blocks a layout scan walks: the PDX blocks (each partition ends
// in a padded block) or ceil(n/64) groups of rows / DSM columns.
static int64_t layout_blocks(const pdx_index *ix, int layout) {
    return layout == PDX_LAYOUT_PDX_KERNEL ? ix->nblocks : (ix->n + kBlock - 1) / kBlock;
}

size_t layout_scratch_bytes(const pdx_index *ix, int layout, int64_t nq, int32_t k) {
    const int64_t nchunks = (layout_blocks(ix, layout) + kChunkBlocks - 1) / kChunkBlocks;
    auto rup = [](size_t b) { return (b + 255) & ~size_t(255); };
    return rup((size_t)nq * nchunks * k * 8) + 3 * rup((size_t)nq * k * 8) + rup(8);
}

pdx_status layout_run(const pdx_index *ix, const float *qd, int64_t nq, int32_t k, int layout, int metric,
                      int out_mode, unsigned char *scratch, float *od, int64_t *oi, int sms, void *ev_start,
                      void *ev_stop, cudaStream_t st) {
    const int64_t nblk = layout_blocks(ix, layout);
    const int64_t nchunks = (nblk + kChunkBlocks - 1) / kChunkBlocks;
    auto rup = [](size_t b) { return (b + 255) & ~size_t(255); };
    size_t off = 0;
    uint64_t *cand = reinterpret_cast<uint64_t *>(scratch + off);
    off += rup((size_t)nq * nchunks * k * 8);
    uint64_t *topk = reinterpret_cast<uint64_t *>(scratch + off);
    off += rup((size_t)nq * k * 8);
    uint64_t *refined = reinterpret_cast<uint64_t *>(scratch + off);
    off += rup((size_t)nq * k * 8);
    uint64_t *final_keys = reinterpret_cast<uint64_t *>(scratch + off);
    off += rup((size_t)nq * k * 8);
    int *work = reinterpret_cast<int *>(scratch + off);
    cudaError_t e = cudaMemsetAsync(work, 0, 8, st);
    if (e != cudaSuccess) return cuda_status_ext(e, "layout scan");
    LayoutParams p;
    std::memset(&p, 0, sizeof p);
    p.layout = layout;
    p.x = layout == PDX_LAYOUT_PDX_KERNEL ? ix->data : (layout == PDX_LAYOUT_DSM ? ix->dsm : ix->xnary);
    p.ids = ix->ids;
    p.n = ix->n;
    p.n_pad = (ix->n + kBlock - 1) / kBlock * kBlock;
    p.nblk = nblk;
    p.d = ix->d;
    p.q = qd;
    p.nq = nq;
    p.k = k;
    p.nchunks = nchunks;
    p.cand = cand;
    p.work_counter = work;
    p.nitems = nq * nchunks;
    const size_t smem = (size_t)kLayoutWarps * warp_bytes(layout, ix->d, k);
    int per_sm = 1;
    switch (layout) {
    case PDX_LAYOUT_PDX_KERNEL:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, layout_scan_kernel<MT_L2, PDX_LAYOUT_PDX_KERNEL>,
                                                      kLayoutWarps * 32, smem);
        break;
    case PDX_LAYOUT_DSM:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, layout_scan_kernel<MT_L2, PDX_LAYOUT_DSM>,
                                                      kLayoutWarps * 32, smem);
        break;
    case PDX_LAYOUT_NARY:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, layout_scan_kernel<MT_L2, PDX_LAYOUT_NARY>,
                                                      kLayoutWarps * 32, smem);
        break;
    default:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, layout_scan_kernel<MT_L2, PDX_LAYOUT_NARY_GATHER>,
                                                      kLayoutWarps * 32, smem);
    }
    cudaGetLastError();
    if (per_sm < 1) per_sm = 1;
    const int64_t want = (p.nitems + kLayoutWarps - 1) / kLayoutWarps;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * per_sm, want));
    if (ev_start && (e = cudaEventRecord(static_cast<cudaEvent_t>(ev_start), st)) != cudaSuccess)
        return cuda_status_ext(e, "layout scan");
    switch (layout) {
    case PDX_LAYOUT_PDX_KERNEL: e = launch_layout_t<PDX_LAYOUT_PDX_KERNEL>(metric, p, smem, grid, st); break;
    case PDX_LAYOUT_DSM: e = launch_layout_t<PDX_LAYOUT_DSM>(metric, p, smem, grid, st); break;
    case PDX_LAYOUT_NARY: e = launch_layout_t<PDX_LAYOUT_NARY>(metric, p, smem, grid, st); break;
    default: e = launch_layout_t<PDX_LAYOUT_NARY_GATHER>(metric, p, smem, grid, st);
    }
    if (e != cudaSuccess) return cuda_status_ext(e, "layout scan");
    if (ev_stop && (e = cudaEventRecord(static_cast<cudaEvent_t>(ev_stop), st)) != cudaSuccess)
        return cuda_status_ext(e, "layout scan");
    // merge the per-item lists, canonical distances, output (as the PDX scan)
    if ((e = launch_select_k(cand, nq, nchunks * k, k, topk, st)) != cudaSuccess)
        return cuda_status_ext(e, "layout scan merge");
    if (ix->xnary && ix->metric != PDX_L1)
        e = launch_refine_rows(topk, nq, k, qd, ix->d, ix->xnary, ix->metric, refined, st);
    else
        e = launch_refine(topk, nq, k, qd, ix->d, ix->data, ix->slot_of, ix->metric, refined, st);
    if (e != cudaSuccess) return cuda_status_ext(e, "layout scan refine");
    if ((e = launch_select_k(refined, nq, k, k, final_keys, st)) != cudaSuccess)
        return cuda_status_ext(e, "layout scan output");
    if ((e = launch_write_out(final_keys, nq, k, out_mode, qd, ix->d, od, oi, st)) != cudaSuccess)
        return cuda_status_ext(e, "layout scan output");
    return PDX_OK;
}

}  // namespace pdx
