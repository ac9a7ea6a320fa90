// The kernels around the PDXearch scan: START keys (exact distances of the
// first vectors, the start-cluster centroids and their members), k-smallest
// selection, canonical refinement of the results, visit orders (Sec. 5) and
// the fused pruner's distance mass.
#include <algorithm>

#include "pdx_internal.cuh"

namespace pdx {

// ---------------------------------------------------------------------------
// START (Sec. 4, PHASE 0) for exact search and the IVF bucket search: exact
// distances of a tile of 128 queries to one 64-vector block, fully over D,
// written as (distance, id) keys. Each thread owns 8 queries x 4 vectors; the
// block's dimension slices are already dimension-major in PDX order and are
// staged 16 dimensions at a time, the next 16 loaded into registers while the
// current ones are used. Every distance is summed in dimension order.
template <int MET>
__global__ void __launch_bounds__(256) dense_keys_kernel(const float *__restrict__ q, int64_t nq,
                                                         const float *__restrict__ data,
                                                         const int32_t *__restrict__ ids, int32_t d, int32_t nblk,
                                                         uint64_t *__restrict__ keys) {
    constexpr int TQ = 128, KC = 16;
    __shared__ __align__(16) float Qs[KC][TQ + 4];  // [dimension][query], padded rows
    __shared__ __align__(16) float Xs[KC][kBlock];  // [dimension][vector]: the block's own layout
    const int tid = threadIdx.x;
    const int64_t q0 = (int64_t)blockIdx.x * TQ;
    const int b = blockIdx.y;
    const int ty = tid >> 4, tx = tid & 15;  // queries ty*8..+7, vectors tx*4..+3
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    const float *xb = data + (int64_t)b * d * kBlock;
    // the next chunk is loaded into registers while the current one is used
    float qpf[8];
    float4 xpf;
    auto load = [&](int j0) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = tid + 256 * u;
            const int qq = e >> 4, jj = e & 15;
            const int64_t qi = q0 + qq;
            qpf[u] = (qi < nq && j0 + jj < d) ? q[qi * d + j0 + jj] : 0.f;
        }
        const int jj = tid >> 4;
        xpf = (j0 + jj < d) ? *reinterpret_cast<const float4 *>(xb + (int64_t)(j0 + jj) * kBlock + (tid & 15) * 4)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    load(0);
    for (int j0 = 0; j0 < d; j0 += KC) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = tid + 256 * u;
            Qs[e & 15][e >> 4] = qpf[u];
        }
        *reinterpret_cast<float4 *>(&Xs[tid >> 4][(tid & 15) * 4]) = xpf;
        __syncthreads();
        if (j0 + KC < d) load(j0 + KC);
        const int jn = min(KC, d - j0);
        for (int jj = 0; jj < jn; ++jj) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&Qs[jj][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&Qs[jj][ty * 8 + 4]);
            const float4 bv = *reinterpret_cast<const float4 *>(&Xs[jj][tx * 4]);
            const float aa[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = term<MET>(aa[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
    const int64_t L = (int64_t)nblk * kBlock;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t qi = q0 + ty * 8 + i;
        if (qi >= nq) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int v = tx * 4 + j;
            const int32_t id = ids[(int64_t)b * kBlock + v];
            keys[qi * L + (int64_t)b * kBlock + v] = (id >= 0) ? make_key(rank_dist<MET>(acc[i][j]), id) : kEmptyKey;
        }
    }
}

// START on row-major FP32 vectors (the low-precision indexes' FP32 copy, and
// the start-cluster centroids): keys[qi][r] = (exact distance of row r, id r)
// for the first nrows rows, the empty key for nrows <= r < ld. A CTA computes a 32 x 32 tile (2 x 2 per thread)
// so that even 1000 queries x 244 centroids spread over the SMs; the shared
// tiles are padded to 33 columns for conflict-free transposed stores.
__global__ void __launch_bounds__(256) dense_keys_rows_kernel(const float *__restrict__ q, int64_t nq,
                                                              const float *__restrict__ x, int32_t nrows, int32_t d,
                                                              int64_t ld, uint64_t *__restrict__ keys) {
    __shared__ float Qs[32][33];
    __shared__ float Xs[32][33];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int64_t q0 = (int64_t)blockIdx.x * 32;
    const int r0 = blockIdx.y * 32;
    float acc[2][2] = {};
    for (int j0 = 0; j0 < d; j0 += 32) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = tid + 256 * u;
            const int rr = e >> 5, jj = e & 31;
            const int j = j0 + jj;
            const int64_t qi = q0 + rr;
            Qs[jj][rr] = (qi < nq && j < d) ? q[qi * d + j] : 0.f;
            const int r = r0 + rr;
            Xs[jj][rr] = (r < nrows && j < d) ? x[(int64_t)r * d + j] : 0.f;
        }
        __syncthreads();
        const int jn = min(32, d - j0);
        for (int jj = 0; jj < jn; ++jj) {
            const float a0 = Qs[jj][ty * 2], a1 = Qs[jj][ty * 2 + 1];
            const float b0 = Xs[jj][tx * 2], b1 = Xs[jj][tx * 2 + 1];
            float t = a0 - b0;
            acc[0][0] = fmaf(t, t, acc[0][0]);
            t = a0 - b1;
            acc[0][1] = fmaf(t, t, acc[0][1]);
            t = a1 - b0;
            acc[1][0] = fmaf(t, t, acc[1][0]);
            t = a1 - b1;
            acc[1][1] = fmaf(t, t, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int64_t qi = q0 + ty * 2 + i;
        if (qi >= nq) continue;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int r = r0 + tx * 2 + j;
            if (r < ld) keys[qi * ld + r] = (r < nrows) ? make_key(acc[i][j], r) : kEmptyKey;
        }
    }
}

cudaError_t launch_dense_keys_rows(const float *q, int64_t nq, const float *x, int32_t nrows, int32_t d, int64_t ld,
                                   uint64_t *keys, cudaStream_t st) {
    if (nq == 0 || nrows == 0) return cudaSuccess;
    if (nrows > ld) return cudaErrorInvalidValue;
    // the tiles cover all ld columns, so the padding keys are written too
    dim3 grid((unsigned)((nq + 31) / 32), (unsigned)((ld + 31) / 32));
    dense_keys_rows_kernel<<<grid, 256, 0, st>>>(q, nq, x, nrows, d, ld, keys);
    return counted(cudaGetLastError());
}

// START from the query's nearest start clusters: a warp per (query, member)
// vector, exact FP32 L2 from the row-major vectors (16-byte pieces, eight in
// flight per lane, when d is a multiple of 4 and the rows are aligned), or
// from the PDX blocks through slot_of when the index keeps no rows.
// keys[qi][p*M + m] = (distance, id) of member m of the query's p-th nearest
// cluster (empty for padding). Each vector belongs to one cluster, so the keys
// are distinct vectors and their k-th smallest distance bounds the final k-th
// from above.
__global__ void member_keys_kernel(const float *__restrict__ q, int64_t nq, int32_t d, const float *__restrict__ rows,
                                   const float *__restrict__ data, const int32_t *__restrict__ slot_of,
                                   const uint64_t *__restrict__ nearest, int32_t P, const int32_t *__restrict__ members,
                                   int32_t M, int vec4, uint64_t *__restrict__ keys) {
    const int64_t qi = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const int e = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (qi >= nq || e >= P * M) return;
    const int p = e / M, m = e % M;
    const uint64_t ck = nearest[qi * P + p];
    const int32_t id = (ck != kEmptyKey) ? members[(int64_t)key_id(ck) * M + m] : -1;
    uint64_t key = kEmptyKey;
    if (id >= 0) {
        const float *qrow = q + qi * d;
        float acc = 0.f;
        if (rows && vec4) {
            const float4 *x4 = reinterpret_cast<const float4 *>(rows + (int64_t)id * d);
            const float4 *q4 = reinterpret_cast<const float4 *>(qrow);
            const int n4 = d >> 2;
            for (int base = lane; base < n4; base += 256) {
                float4 xv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    xv[u] = (base + 32 * u < n4) ? __ldg(x4 + base + 32 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (base + 32 * u < n4) {
                        const float4 qv = __ldg(q4 + base + 32 * u);
                        acc = term<MT_L2>(qv.x, xv[u].x, acc);
                        acc = term<MT_L2>(qv.y, xv[u].y, acc);
                        acc = term<MT_L2>(qv.z, xv[u].z, acc);
                        acc = term<MT_L2>(qv.w, xv[u].w, acc);
                    }
                }
            }
        } else if (rows) {
            const float *xr = rows + (int64_t)id * d;
            for (int j = lane; j < d; j += 32) acc = term<MT_L2>(qrow[j], __ldg(xr + j), acc);
        } else {
            const int32_t slot = slot_of[id];
            const float *xb = data + (int64_t)(slot / kBlock) * d * kBlock + (slot % kBlock);
            for (int j = lane; j < d; j += 32) acc = term<MT_L2>(qrow[j], __ldg(xb + (int64_t)j * kBlock), acc);
        }
        key = make_key(warp_sum(acc), id);
    }
    if (lane == 0) keys[qi * (int64_t)P * M + e] = key;
}

cudaError_t launch_member_keys(const float *q, int64_t nq, int32_t d, const float *rows, const float *data,
                               const int32_t *slot_of, const uint64_t *nearest, int32_t P, const int32_t *members,
                               int32_t M, uint64_t *keys, cudaStream_t st) {
    if (nq == 0 || P * M == 0) return cudaSuccess;
    const int vec4 = (d % 4 == 0 && ((uintptr_t)rows & 15u) == 0 && ((uintptr_t)q & 15u) == 0) ? 1 : 0;
    dim3 grid((unsigned)nq, (unsigned)((P * M + 7) / 8));
    member_keys_kernel<<<grid, 256, 0, st>>>(q, nq, d, rows, data, slot_of, nearest, P, members, M, vec4, keys);
    return counted(cudaGetLastError());
}

cudaError_t launch_dense_keys(const float *q, int64_t nq, const float *data, const int32_t *ids, int32_t d,
                              int32_t nblk, int metric, uint64_t *keys, cudaStream_t st) {
    if (nq == 0 || nblk == 0) return cudaSuccess;
    dim3 grid((unsigned)((nq + 127) / 128), (unsigned)nblk);
    if (metric == MT_IP)
        dense_keys_kernel<MT_IP><<<grid, 256, 0, st>>>(q, nq, data, ids, d, nblk, keys);
    else if (metric == MT_L1)
        dense_keys_kernel<MT_L1><<<grid, 256, 0, st>>>(q, nq, data, ids, d, nblk, keys);
    else
        dense_keys_kernel<MT_L2><<<grid, 256, 0, st>>>(q, nq, data, ids, d, nblk, keys);
    return counted(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// k smallest keys of each row: the row is consumed in chunks appended after the
// running best kpad keys and the buffer is bitonic-sorted by the whole CTA.
__global__ void __launch_bounds__(512) select_k_kernel(const uint64_t *__restrict__ keys, int64_t L, int32_t k,
                                                       int32_t kpad, int32_t sb, uint64_t *__restrict__ out) {
    extern __shared__ __align__(16) uint64_t buf[];
    const int64_t row = blockIdx.x;
    const uint64_t *src = keys + row * L;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < kpad; i += nt) buf[i] = kEmptyKey;
    const int chunk = sb - kpad;
    for (int64_t off = 0; off < L; off += chunk) {
        for (int i = tid; i < chunk; i += nt) buf[kpad + i] = (off + i < L) ? src[off + i] : kEmptyKey;
        __syncthreads();
        for (int size = 2; size <= sb; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = tid; i < (sb >> 1); i += nt) {
                    int lo = 2 * i - (i & (stride - 1));
                    int hi = lo + stride;
                    bool asc = (lo & size) == 0;
                    uint64_t x = buf[lo], y = buf[hi];
                    if ((x > y) == asc) {
                        buf[lo] = y;
                        buf[hi] = x;
                    }
                }
                __syncthreads();
            }
        }
    }
    for (int i = tid; i < k; i += nt) out[row * k + i] = buf[i];
}

// k <= 8 smallest keys of each row, a warp per row: every lane keeps the
// smallest keys of its stride of the row in a sorted register list, then k
// rounds of a warp-wide minimum pop them in order.
__global__ void select_small_kernel(const uint64_t *__restrict__ keys, int64_t rows, int64_t L, int32_t k,
                                    uint64_t *__restrict__ out) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    uint64_t best[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) best[i] = kEmptyKey;
    const uint64_t *kr = keys + row * L;
    for (int64_t i = lane; i < L; i += 32) {
        uint64_t v = kr[i];
        if (v >= best[7]) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {  // insertion into the sorted list
            const uint64_t lo = v < best[j] ? v : best[j];
            v = v < best[j] ? best[j] : v;
            best[j] = lo;
        }
    }
    for (int r = 0; r < k; ++r) {
        uint64_t m = best[0];
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const uint64_t t = __shfl_xor_sync(kFull, m, o);
            m = t < m ? t : m;
        }
        // the lane holding the minimum (the lowest such lane) pops it
        const unsigned own = __ballot_sync(kFull, best[0] == m);
        if (lane == __ffs(own) - 1) {
#pragma unroll
            for (int j = 0; j < 7; ++j) best[j] = best[j + 1];
            best[7] = kEmptyKey;
        }
        if (lane == 0) out[row * k + r] = m;
    }
}

cudaError_t launch_select_k(const uint64_t *keys, int64_t rows, int64_t L, int32_t k, uint64_t *out,
                            cudaStream_t st) {
    if (rows == 0) return cudaSuccess;
    if (k <= 8 && L <= 4096) {  // a warp per row
        select_small_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(keys, rows, L, k, out);
        return counted(cudaGetLastError());
    }
    int kpad = pow2_ceil(k);
    int64_t want = (int64_t)kpad + L;
    int sb = pow2_ceil((int)(want < 8192 ? want : 8192));
    if (sb < 2 * kpad) sb = 2 * kpad;
    if (sb < 64) sb = 64;
    size_t smem = (size_t)sb * 8;
    cudaError_t e = raise_smem_limit(select_k_kernel, smem);
    if (e != cudaSuccess) return e;
    int threads = sb >= 1024 ? 512 : (sb / 2 < 32 ? 32 : sb / 2);
    select_k_kernel<<<(unsigned)rows, threads, smem, st>>>(keys, L, k, kpad, sb, out);
    return counted(cudaGetLastError());
}

// k smallest keys of each row whose distance is within the row's final
// threshold: tau[row] is the k-th distance of k real vectors found by the
// scan, so the k smallest keys are all within slack(tau, gamma) (the slack
// covers FP32 sums taken in another order, e.g. by START). Keys within it are
// compacted into shared memory and sorted. A row with more of them than the
// buffer holds (a scan whose threshold tightened late, e.g. one query spread
// over many work items in one wave) takes the k-th smallest of the sb keys it
// kept as its new limit: that is the k-th distance of k real candidates, so it
// still bounds the row's k-th from above, and the row is filtered again. If a
// round brings no progress (ties) the chunked sort of select_k_kernel decides.
__device__ __forceinline__ void block_bitonic(uint64_t *buf, int len, int tid, int nt) {
    for (int size = 2; size <= len; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < (len >> 1); i += nt) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool asc = (lo & size) == 0;
                const uint64_t x = buf[lo], y = buf[hi];
                if ((x > y) == asc) {
                    buf[lo] = y;
                    buf[hi] = x;
                }
            }
            __syncthreads();
        }
    }
}

// Small batches: one row's keys are filtered by many CTAs (slices of the row)
// into a compact per-row buffer of `cap` keys, with a per-row counter
// (zeroed before the launch). A row whose keys within the limit exceed cap
// is selected from its full row instead.
__global__ void __launch_bounds__(512) filter_keys_kernel(const uint64_t *__restrict__ keys, int64_t L,
                                                          const float *__restrict__ tau, float gamma, int32_t cap,
                                                          uint64_t *__restrict__ compact, int32_t *__restrict__ counts) {
    const int64_t row = blockIdx.y;
    const int64_t per = (L + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * per;
    const int64_t hi = min(L, lo + per);
    const uint64_t *src = keys + row * L;
    const float t = o2f(reinterpret_cast<const uint32_t *>(tau)[row]);
    const uint32_t lim = f2o(t + fabsf(t) * gamma);
    const int nt = blockDim.x;
    for (int64_t base = lo + threadIdx.x; base < hi; base += (int64_t)nt * 8) {
        uint64_t kk[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t i = base + (int64_t)u * nt;
            kk[u] = i < hi ? src[i] : kEmptyKey;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (kk[u] != kEmptyKey && (uint32_t)(kk[u] >> 32) <= lim) {
                const int pos = atomicAdd(counts + row, 1);
                if (pos < cap) compact[row * cap + pos] = kk[u];
            }
        }
    }
}

__global__ void __launch_bounds__(512) select_k_tau_kernel(const uint64_t *__restrict__ keys, int64_t L, int32_t k,
                                                           const float *__restrict__ tau, float gamma, int32_t sb,
                                                           const uint64_t *__restrict__ compact,
                                                           const int32_t *__restrict__ counts, int32_t cap,
                                                           uint64_t *__restrict__ out) {
    extern __shared__ __align__(16) uint64_t buf[];
    __shared__ int count;
    const int64_t row = blockIdx.x;
    const uint64_t *src = keys + row * L;
    if (counts) {   // filtered by filter_keys_kernel: its compact keys, unless they overflowed
        const int c = counts[row];
        if (c <= cap) {
            src = compact + row * cap;
            L = c;
        }
    }
    const int tid = threadIdx.x, nt = blockDim.x;
    const float t = o2f(reinterpret_cast<const uint32_t *>(tau)[row]);
    uint32_t lim = f2o(t + fabsf(t) * gamma);
    for (int round = 0; round < 4; ++round) {
        if (tid == 0) count = 0;
        __syncthreads();
        // eight independent loads in flight per thread: a small batch leaves
        // one CTA to read a long row (1 query: every work item's list)
        for (int64_t base = tid; base < L; base += (int64_t)nt * 8) {
            uint64_t kk[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t i = base + (int64_t)u * nt;
                kk[u] = i < L ? src[i] : kEmptyKey;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (kk[u] != kEmptyKey && (uint32_t)(kk[u] >> 32) <= lim) {
                    const int pos = atomicAdd(&count, 1);
                    if (pos < sb) buf[pos] = kk[u];
                }
            }
        }
        __syncthreads();
        const int c = count;
        const int m = c < sb ? c : sb;
        int len = 1;
        while (len < (m > k ? m : k)) len <<= 1;   // <= sb: sb is a power of two >= 2 * pow2(k)
        for (int i = m + tid; i < len; i += nt) buf[i] = kEmptyKey;
        __syncthreads();
        block_bitonic(buf, len, tid, nt);
        if (c <= sb) {
            for (int i = tid; i < k; i += nt) out[row * k + i] = buf[i];
            return;
        }
        const uint32_t nl = (uint32_t)(buf[k - 1] >> 32);   // m = sb >= k real keys
        __syncthreads();
        if (nl >= lim) break;
        lim = nl;
    }
    // fallback: running best kpad of all keys, chunks appended and sorted
    int kpad = 1;
    while (kpad < k) kpad <<= 1;
    for (int i = tid; i < kpad; i += nt) buf[i] = kEmptyKey;
    const int chunk = sb - kpad;
    for (int64_t off = 0; off < L; off += chunk) {
        __syncthreads();
        for (int i = tid; i < chunk; i += nt) buf[kpad + i] = (off + i < L) ? src[off + i] : kEmptyKey;
        __syncthreads();
        block_bitonic(buf, sb, tid, nt);
    }
    for (int i = tid; i < k; i += nt) out[row * k + i] = buf[i];
}

cudaError_t launch_select_k_tau(const uint64_t *keys, int64_t rows, int64_t L, int32_t k, const float *tau,
                                float gamma, uint64_t *out, cudaStream_t st, uint64_t *compact, int32_t *counts) {
    if (rows == 0) return cudaSuccess;
    int kpad = pow2_ceil(k);
    const int sb = std::max(kSplitSelectCap, 2 * kpad);  // power of two (kpad <= 1024)
    const size_t smem = (size_t)sb * 8;
    cudaError_t e = raise_smem_limit(select_k_tau_kernel, smem);
    if (e != cudaSuccess) return e;
    const bool split = compact && counts && rows <= kSplitSelectRows && L > 4096 && sb == kSplitSelectCap;
    if (split) {
        // 128 slices in all, whatever the batch (1 query: 128 CTAs over its row)
        const int slices = (int)std::max<int64_t>(1, std::min<int64_t>(128 / rows, (L + 4095) / 4096));
        e = cudaMemsetAsync(counts, 0, (size_t)rows * 4, st);
        if (e != cudaSuccess) return e;
        filter_keys_kernel<<<dim3((unsigned)slices, (unsigned)rows), 512, 0, st>>>(keys, L, tau, gamma,
                                                                                   kSplitSelectCap, compact, counts);
        e = counted(cudaGetLastError());
        if (e != cudaSuccess) return e;
    }
    select_k_tau_kernel<<<(unsigned)rows, 512, smem, st>>>(keys, L, k, tau, gamma, sb, split ? compact : nullptr,
                                                            split ? counts : nullptr, kSplitSelectCap, out);
    return counted(cudaGetLastError());
}

__global__ void tau_from_keys_kernel(const uint64_t *topk, int64_t rows, int32_t k, float *tau) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    uint64_t key = topk[r * k + k - 1];
    uint32_t v = (key == kEmptyKey) ? f2o(__int_as_float(0x7f800000)) : f2o(key_dist(key));
    reinterpret_cast<uint32_t *>(tau)[r] = v;
}

cudaError_t launch_tau_from_keys(const uint64_t *topk, int64_t rows, int32_t k, float *tau, cudaStream_t st) {
    if (rows == 0) return cudaSuccess;
    tau_from_keys_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(topk, rows, k, tau);
    return counted(cudaGetLastError());
}

__global__ void tau_min_kernel(float *tau, const float *init, int64_t rows) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    uint32_t *t = reinterpret_cast<uint32_t *>(tau) + r;
    const float v = init[r];
    const uint32_t o = (v != v) ? f2o(__int_as_float(0x7f800000)) : f2o(v);  // NaN: no bound
    if (o < *t) *t = o;
}

cudaError_t launch_tau_min(float *tau, const float *init, int64_t rows, cudaStream_t st) {
    if (rows == 0) return cudaSuccess;
    tau_min_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(tau, init, rows);
    return counted(cudaGetLastError());
}

// One warp per (query, result): lanes take dimensions j = lane, lane+32, ...
// of the vector's storage slot, then a fixed butterfly reduction. Identical
// vectors therefore get bit-identical distances, whatever order the scan
// visited their dimensions in, and ties order by id.
template <int MET>
__global__ void refine_kernel(const uint64_t *__restrict__ topk, int64_t nq, int32_t k, const float *__restrict__ q,
                              int32_t d, const float *__restrict__ data, const int32_t *__restrict__ slot_of,
                              uint64_t *__restrict__ out) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nq * k) return;
    const int64_t row = w / k;
    const uint64_t key = topk[w];
    if (key == kEmptyKey) {
        if (lane == 0) out[w] = kEmptyKey;
        return;
    }
    const int32_t id = key_id(key);
    const int32_t slot = slot_of[id];
    const float *xb = data + (int64_t)(slot / kBlock) * d * kBlock + (slot % kBlock);
    const float *qr = q + row * d;
    float acc = 0.f;
    for (int j = lane; j < d; j += 32) acc = term<MET>(qr[j], xb[(int64_t)j * kBlock], acc);
    acc = warp_sum(acc);
    if (lane == 0) out[w] = make_key(rank_dist<MET>(acc), id);
}

// Canonical distances from row-major FP32 vectors (low-precision indexes).
template <int MET>
__global__ void refine_rows_kernel(const uint64_t *__restrict__ topk, int64_t nq, int32_t k, const float *__restrict__ q,
                                   int32_t d, const float *__restrict__ x, uint64_t *__restrict__ out) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nq * k) return;
    const int64_t row = w / k;
    const uint64_t key = topk[w];
    if (key == kEmptyKey) {
        if (lane == 0) out[w] = kEmptyKey;
        return;
    }
    const int32_t id = key_id(key);
    const float *xr = x + (int64_t)id * d;
    const float *qr = q + row * d;
    float acc = 0.f;
    for (int j = lane; j < d; j += 32) acc = term<MET>(qr[j], xr[j], acc);
    acc = warp_sum(acc);
    if (lane == 0) out[w] = make_key(rank_dist<MET>(acc), id);
}

cudaError_t launch_refine_rows(const uint64_t *topk, int64_t nq, int32_t k, const float *q, int32_t d, const float *x,
                               int metric, uint64_t *out, cudaStream_t st) {
    int64_t warps = nq * k;
    if (warps == 0) return cudaSuccess;
    unsigned grid = (unsigned)((warps * 32 + 255) / 256);
    if (metric == MT_IP)
        refine_rows_kernel<MT_IP><<<grid, 256, 0, st>>>(topk, nq, k, q, d, x, out);
    else
        refine_rows_kernel<MT_L2><<<grid, 256, 0, st>>>(topk, nq, k, q, d, x, out);
    return counted(cudaGetLastError());
}

cudaError_t launch_refine(const uint64_t *topk, int64_t nq, int32_t k, const float *q, int32_t d, const float *data,
                          const int32_t *slot_of, int metric, uint64_t *out, cudaStream_t st) {
    int64_t warps = nq * k;
    if (warps == 0) return cudaSuccess;
    unsigned grid = (unsigned)((warps * 32 + 255) / 256);
    if (metric == MT_IP)
        refine_kernel<MT_IP><<<grid, 256, 0, st>>>(topk, nq, k, q, d, data, slot_of, out);
    else if (metric == MT_L1)
        refine_kernel<MT_L1><<<grid, 256, 0, st>>>(topk, nq, k, q, d, data, slot_of, out);
    else
        refine_kernel<MT_L2><<<grid, 256, 0, st>>>(topk, nq, k, q, d, data, slot_of, out);
    return counted(cudaGetLastError());
}

__global__ void write_out_kernel(const uint64_t *topk, int64_t nq, int32_t k, int mode, const float *q, int32_t d,
                                 float *out_dist, int64_t *out_idx) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= nq) return;
    float qn = 0.f;
    if (mode == 2) {
        for (int j = lane; j < d; j += 32) qn = fmaf(q[row * d + j], q[row * d + j], qn);
        qn = warp_sum(qn);
    }
    for (int i = lane; i < k; i += 32) {
        uint64_t key = topk[row * k + i];
        float dist;
        int64_t id;
        if (key == kEmptyKey) {
            id = -1;
            dist = (mode == 0) ? __int_as_float(0x7f800000) : __int_as_float(0xff800000);
        } else {
            id = key_id(key);
            float kd = key_dist(key);
            dist = (mode == 0) ? kd : (mode == 1) ? -kd : 0.5f * (qn + 1.f - kd);
        }
        out_dist[row * k + i] = dist;
        out_idx[row * k + i] = id;
    }
}

cudaError_t launch_write_out(const uint64_t *topk, int64_t nq, int32_t k, int mode, const float *q, int32_t d,
                             float *out_dist, int64_t *out_idx, cudaStream_t st) {
    if (nq == 0) return cudaSuccess;
    write_out_kernel<<<(unsigned)((nq * 32 + 255) / 256), 256, 0, st>>>(topk, nq, k, mode, q, d, out_dist, out_idx);
    return counted(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Query preprocessing for PDX-BOND (Sec. 5): the dimension visit order of each
// row (a query, or a (query, part) pair when per_part > 0), computed once and
// stored as uint16 dimension indices. mode 0: distance to the means (zones of
// Z dimensions, score = sum (q_j - mu_j)^2); mode 1: decreasing query value;
// mode 2: decreasing (q_j - mu_j)^2 + s_q scores[row][j] (the network's
// correction in units of s_q = mean_j (q_j - mu_j)^2).
// One CTA per row sorts its keys (score descending, index ascending) with a
// block-wide bitonic sort in shared memory.
__global__ void __launch_bounds__(256) order_kernel(const float *__restrict__ q, int64_t rows, int32_t d,
                                                    const float *__restrict__ means, int32_t per_part,
                                                    const int32_t *__restrict__ row_part, int mode, int32_t Z,
                                                    const float *__restrict__ scores, uint16_t *__restrict__ out) {
    extern __shared__ __align__(16) uint64_t keys[];
    const int64_t row = blockIdx.x;
    if (row >= rows) return;
    const int64_t qi = per_part > 0 ? row / per_part : row;
    const float *qrow = q + qi * d;
    int part = 0;
    if (per_part > 0) part = row_part ? row_part[row] : (int)(row % per_part);
    if (part < 0) part = 0;   // unused probe slot: any valid row of means
    const float *mu = means + (int64_t)part * d;
    const int nunits = (mode >= 1) ? d : (d + Z - 1) / Z;
    const int zz = (mode >= 1) ? 1 : Z;
    const int npad = pow2_ceil(nunits);
    // learned order: the network's outputs are in units of this query's mean
    // heuristic term s_q = mean_j (q_j - mu_j)^2
    __shared__ float sq_part[256];
    float sq = 0.f;
    if (mode == 2) {
        float part = 0.f;
        for (int j = threadIdx.x; j < d; j += blockDim.x) {
            float t = qrow[j] - mu[j];
            part = fmaf(t, t, part);
        }
        sq_part[threadIdx.x] = part;
        __syncthreads();
        for (int o = blockDim.x >> 1; o; o >>= 1) {
            if ((int)threadIdx.x < o) sq_part[threadIdx.x] += sq_part[threadIdx.x + o];
            __syncthreads();
        }
        sq = sq_part[0] / (float)d;
    }
    for (int u = threadIdx.x; u < npad; u += blockDim.x) {
        uint64_t key = kEmptyKey;
        if (u < nunits) {
            float sc = 0.f;
            if (mode == 2) {
                // learned: heuristic (q_j - mu_j)^2 plus the network's correction
                float t = qrow[u] - mu[u];
                sc = fmaf(t, t, sq * scores[row * (int64_t)d + u]);
            } else if (mode == 1) {
                sc = qrow[u];
            } else {
                int j1 = min(d, u * zz + zz);
                for (int j = u * zz; j < j1; ++j) {
                    float t = qrow[j] - mu[j];
                    sc = fmaf(t, t, sc);
                }
            }
            key = ((uint64_t)f2o(-sc) << 32) | (uint32_t)u;
        }
        keys[u] = key;
    }
    __syncthreads();
    for (int size = 2; size <= npad; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < (npad >> 1); i += blockDim.x) {
                int lo = 2 * i - (i & (stride - 1));
                int hi = lo + stride;
                bool asc = (lo & size) == 0;
                uint64_t a = keys[lo], b = keys[hi];
                if ((a > b) == asc) {
                    keys[lo] = b;
                    keys[hi] = a;
                }
            }
            __syncthreads();
        }
    }
    // expand zones: rank r's dimensions start at r*Z, shifted back by the
    // shortfall of the last (shorter) zone when it ranks before r
    __shared__ int rlast;
    if (threadIdx.x == 0) rlast = 0;
    __syncthreads();
    for (int r = threadIdx.x; r < nunits; r += blockDim.x)
        if ((int)(keys[r] & 0xffffffffu) == nunits - 1) rlast = r;
    __syncthreads();
    const int lastlen = d - (nunits - 1) * zz;
    uint16_t *orow = out + row * (int64_t)d;
    for (int r = threadIdx.x; r < nunits; r += blockDim.x) {
        int z = (int)(keys[r] & 0xffffffffu);
        int off = r * zz - ((r > rlast) ? (zz - lastlen) : 0);
        int len = (z == nunits - 1) ? lastlen : zz;
        for (int u = 0; u < len; ++u) orow[off + u] = (uint16_t)(z * zz + u);
    }
}

// F_q(d) of the fused pruner (ADSampling with PDX-BOND's order): for each
// (query, probed bucket) row, E_j = (q_j - mu_j)^2 + var_j is the expected
// (q_j - x_j)^2 of a vector of the bucket, and out[row][c] is the sum of E over
// the first chk[c] dimensions of the row's visit order divided by the sum of E
// over all dimensions. One warp per row.
__global__ void mass_kernel(const float *__restrict__ q, int64_t rows, int32_t d, int32_t per_part,
                            const int32_t *__restrict__ row_part, const float *__restrict__ means,
                            const float *__restrict__ vars, const uint16_t *__restrict__ order,
                            const int32_t *__restrict__ chk, int32_t nchk, float *__restrict__ out) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const int64_t qi = row / per_part;
    const int part = row_part[row];
    float s[kMaxChecks];
    int cp[kMaxChecks];
#pragma unroll
    for (int c = 0; c < kMaxChecks; ++c) {
        s[c] = 0.f;
        cp[c] = c < nchk ? chk[c] : 0;
    }
    float total = 0.f;
    if (part >= 0) {
        const float *qrow = q + qi * d, *mu = means + (int64_t)part * d, *vr = vars + (int64_t)part * d;
        const uint16_t *ord = order + row * (int64_t)d;
        for (int i = lane; i < d; i += 32) {
            const int j = ord[i];
            const float t = qrow[j] - mu[j];
            const float e = fmaf(t, t, vr[j]);
            total += e;
#pragma unroll
            for (int c = 0; c < kMaxChecks; ++c)
                if (i < cp[c]) s[c] += e;
        }
    }
    total = warp_sum(total);
#pragma unroll
    for (int c = 0; c < kMaxChecks; ++c) {
        const float v = warp_sum(s[c]);
        if (lane == 0 && c < nchk) out[row * nchk + c] = total > 0.f ? v / total : 1.f;
    }
}

cudaError_t launch_mass(const float *q, int64_t rows, int32_t d, int32_t per_part, const int32_t *row_part,
                        const float *means, const float *vars, const uint16_t *order, const int32_t *chk, int32_t nchk,
                        float *out, cudaStream_t st) {
    if (rows == 0 || nchk == 0) return cudaSuccess;
    if (nchk > kMaxChecks) return cudaErrorInvalidValue;
    mass_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(q, rows, d, per_part, row_part, means, vars,
                                                                     order, chk, nchk, out);
    return counted(cudaGetLastError());
}

cudaError_t launch_order(const float *q, int64_t rows, int32_t d, const float *means, int32_t per_part,
                         const int32_t *row_part, int mode, int32_t Z, const float *scores, uint16_t *out,
                         cudaStream_t st) {
    if (rows == 0) return cudaSuccess;
    const int nunits = (mode >= 1) ? d : (d + Z - 1) / Z;
    size_t smem = (size_t)pow2_ceil(nunits) * 8;
    cudaError_t e = raise_smem_limit(order_kernel, smem);
    if (e != cudaSuccess) return e;
    order_kernel<<<(unsigned)rows, 256, smem, st>>>(q, rows, d, means, per_part, row_part, mode, Z, scores, out);
    return counted(cudaGetLastError());
}

}  // namespace pdx
