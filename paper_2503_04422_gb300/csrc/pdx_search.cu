// PDXearch on the GPU (Sec. 4) with the PDX-BOND (Sec. 5), ADSampling and
// BSA (Sec. 2.3) predicates, over PDX blocks (Sec. 3, Listing 1).
//
// Work decomposition. A work item is (query, PDXearch block): a partition of
// the exact index or a probed IVF bucket (optionally a contiguous group of its
// 64-vector storage blocks). One warp runs one item at a time and pulls the
// next from a global counter; items are numbered block-major, so the warps in
// flight at any moment read the same few partitions for many queries and the
// partition stays in L2 while they do. Inside an item the warp follows the
// paper's phases for every 64-vector block:
//   WARMUP: fetch dimensions in doubling steps for all 64 vectors (lane l holds
//           vectors 4*(l&15)..+3 for the even or odd dimension of each pair, one
//           float4 load per lane per pair of dimensions = 512 contiguous bytes
//           per warp), evaluate the predicate on the partial distances, count
//           survivors with warp ballots.
//   PRUNE:  once survivors < selection_threshold * 64, keep only their
//           positions (<= 16, in registers) and spread the dimensions of each
//           step over the 32 lanes; per-survivor sums are warp-reduced.
//   merge:  survivors' full distances go into the warp's sorted top-k list in
//           shared memory; its k-th distance is the local threshold, published
//           to the query's global threshold with an atomic min.
// Any threshold that is the k-th distance of k real vectors bounds the final
// k-th distance from above, so a stale or partially-tightened threshold never
// prunes a true neighbour (only the amount of pruning depends on timing).
// A relative slack gamma = D * 2^-23 on every threshold covers the rounding of
// FP32 partial sums, so an FP32 partial that exceeds tau*(1+gamma) has an
// exact partial above the exact tau.
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "pdx_internal.cuh"

namespace pdx {

enum { PR_NONE = 0, PR_BOND = 1, PR_ADS = 2, PR_BSA = 3, PR_ADSB = 4, PR_CSIP = 5 };

// ---- storage types of the PDX blocks ----
enum { ST_F32 = 0, ST_BF16 = 1, ST_FP8 = 2 };

template <int ST> struct Elem;
template <> struct Elem<ST_F32> {
    using T = float;
    static __device__ __forceinline__ float4 load4(const T *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
    static __device__ __forceinline__ float load1(const T *p) { return __ldg(p); }
};
template <> struct Elem<ST_BF16> {
    using T = uint16_t;
    static __device__ __forceinline__ float4 load4(const T *p) {
        uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
        return make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u), __uint_as_float(v.y << 16),
                           __uint_as_float(v.y & 0xffff0000u));
    }
    static __device__ __forceinline__ float load1(const T *p) { return __uint_as_float((uint32_t)__ldg(p) << 16); }
};
template <> struct Elem<ST_FP8> {
    using T = uint8_t;
    static __device__ __forceinline__ float2 cvt2(uint32_t two) {
        __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(two & 0xffffu), __NV_E4M3);
        return __half22float2(*reinterpret_cast<const __half2 *>(&h));
    }
    static __device__ __forceinline__ float4 load4(const T *p) {
        uint32_t v = __ldg(reinterpret_cast<const unsigned int *>(p));
        float2 a = cvt2(v), b = cvt2(v >> 16);
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ float load1(const T *p) {
        __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)__ldg(p), __NV_E4M3);
        return __half2float(*reinterpret_cast<const __half *>(&h));
    }
};

// One term of the distance. F32: the exact (q - x)^2 (or IP / L1 term).
// Low-precision storage under an exact pruner (BOND, NONE): a lower bound of
// (q - x)^2 from the stored x_hat and the per-element quantisation bound e
// (|x - x_hat| <= e): max(0, |q - x_hat| - e)^2, with the float32 rounding of
// |q - x_hat| (and of q / s for FP8) folded into a relative slack. For FP8 the
// value is in units of the per-dimension scale s (qv = q/s, s2 = s^2).
// Under an approximate pruner (ADSampling, BSA) the stored value is used as
// is. Survivors of low-precision scans are reranked in FP32.
template <int ST, bool LB>
__device__ __forceinline__ float lp_term(float qv, float xh, float acc, float s2) {
    if (ST == ST_F32 || !LB) {
        float t = qv - xh;
        return (ST == ST_FP8) ? fmaf(s2 * t, t, acc) : fmaf(t, t, acc);
    } else if (ST == ST_BF16) {
        float e = fmaxf(fabsf(xh) * 3.90625607e-3f, 4.6e-41f);           // |x_hat| 2^-8 (1+2^-20), 2^-134
        float t = fabsf(qv - xh) * 0.99999976f - e;                      // (1 - 2^-22)
        return t > 0.f ? fmaf(t, t, acc) : acc;
    } else {
        float e = fmaxf(fabsf(xh) * 6.25006e-2f, 9.765634e-4f);          // max(|c| 2^-4, 2^-10) (1+2^-20)
        float t = fabsf(qv - xh) * 0.99999976f - e - fabsf(qv) * 2.3841858e-7f;
        return t > 0.f ? fmaf(s2 * t, t, acc) : acc;
    }
}

__device__ __forceinline__ float sel4(const float4 &v, int c) {
    return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

__device__ __forceinline__ float slack(float tau, float gamma) { return tau + fabsf(tau) * gamma; }

__device__ __forceinline__ int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Insert `key` into the warp's ascending list (capacity k). Warp-uniform call.
__device__ __forceinline__ void topk_insert(uint64_t *list, int &cnt, int k, uint64_t key, int lane) {
    if (cnt == k && key >= list[k - 1]) return;
    int pos = 0;
    for (int base = 0; base < cnt; base += 32) {
        int i = base + lane;
        bool lt = (i < cnt) && (list[i] < key);
        pos += __popc(__ballot_sync(kFull, lt));
    }
    int newcnt = cnt < k ? cnt + 1 : k;
    int top = newcnt - 1;
    for (int base = (top >> 5) << 5; base >= 0; base -= 32) {
        int i = base + lane;
        bool mv = (i > pos) && (i <= top);
        uint64_t v = mv ? list[i - 1] : 0ull;
        __syncwarp();
        if (mv) list[i] = v;
        __syncwarp();
        if (base <= pos) break;
    }
    if (lane == 0) list[pos] = key;
    __syncwarp();
    cnt = newcnt;
}

struct WarpSmem {
    uint16_t *ord;      // [d] dimension visited at position i
    float *qo;          // [d] query value of that dimension (FP8 storage: divided by its scale)
    float *s2o;         // [d] FP8 storage: squared scale of that dimension
    uint64_t *topk;     // [k]
    int32_t *sv;        // [kMaxSurv] survivor slot indices
    float *sp;          // [kMaxSurv] survivor partial distances
    unsigned long long *ctr;  // [kStats] the warp's statistics; lane 0 adds to them
};

// Statistics a scan warp keeps in shared memory (registers are the scarce
// resource of the scan) and adds to the launch counters when it ends.
enum ScanStat { S_VALUES = 0, S_SCANNED, S_PRUNED, S_PBLOCKS, S_CAND, S_ITEMS, kStats };

// The scan kernel sorts at most kMaxSortUnits zone keys itself, in registers
// (8 per lane); finer orders are computed once per query (or per query and
// part) by order_kernel. Shared memory per warp is kept to 6 bytes per
// dimension: the kernel's loads are latency-bound, and every byte of shared
// memory is taken from the L1 that holds the lines of loads in flight.

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

// Number of zone keys the scan kernel sorts per work item (0 = order given).
__host__ __device__ inline int sort_units(int d, int zone_dims, int order, int pruner, bool given) {
    if (given || pruner != PR_BOND || order != PDX_ORDER_DIST_TO_MEANS) return 0;
    int z = zone_dims < 1 ? 1 : zone_dims;
    return (d + z - 1) / z;
}

__host__ __device__ inline size_t warp_smem_bytes(int d, int k, bool scaled) {
    return align16((size_t)d * 2) + align16((size_t)d * 4) * (scaled ? 2 : 1) + align16((size_t)k * 8) +
           align16(kMaxSurv * 4) * 2 + align16(kStats * 8);
}

size_t scan_warp_smem(int d, int k, int zone_dims, int order) {
    (void)zone_dims;
    (void)order;
    return warp_smem_bytes(d, k, false);
}

__device__ __forceinline__ WarpSmem carve(unsigned char *base, int d, int k, bool scaled) {
    WarpSmem w;
    size_t o = 0;
    w.ord = reinterpret_cast<uint16_t *>(base + o);
    o += align16((size_t)d * 2);
    w.qo = reinterpret_cast<float *>(base + o);
    o += align16((size_t)d * 4);
    w.s2o = nullptr;
    if (scaled) {
        w.s2o = reinterpret_cast<float *>(base + o);
        o += align16((size_t)d * 4);
    }
    w.topk = reinterpret_cast<uint64_t *>(base + o);
    o += align16((size_t)k * 8);
    w.sv = reinterpret_cast<int32_t *>(base + o);
    o += align16(kMaxSurv * 4);
    w.sp = reinterpret_cast<float *>(base + o);
    o += align16(kMaxSurv * 4);
    w.ctr = reinterpret_cast<unsigned long long *>(base + o);
    return w;
}

// Ascending bitonic sort of 32*M keys held in registers, element e = t*32 + lane
// in key[t]: strides >= 32 compare registers of the same lane, strides < 32
// exchange with lane ^ stride.
template <int M>
__device__ __forceinline__ void reg_bitonic_sort(uint64_t (&key)[8], int lane) {
#pragma unroll
    for (int size = 2; size <= 32 * M; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {
                const int ts = stride >> 5;
#pragma unroll
                for (int t = 0; t < M; ++t) {
                    if ((t & ts) == 0) {
                        const int e = t * 32 + lane;
                        const bool asc = (e & size) == 0;
                        uint64_t a = key[t], b = key[t ^ ts];
                        if ((a > b) == asc) {
                            key[t] = b;
                            key[t ^ ts] = a;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int t = 0; t < M; ++t) {
                    const int e = t * 32 + lane;
                    const bool asc = (e & size) == 0;
                    const bool lower = (lane & stride) == 0;
                    uint64_t other = __shfl_xor_sync(kFull, key[t], stride);
                    uint64_t mn = key[t] < other ? key[t] : other;
                    uint64_t mx = key[t] < other ? other : key[t];
                    key[t] = (lower == asc) ? mn : mx;
                }
            }
        }
    }
}

// Visit order of one (query, PDXearch block) work item (Sec. 5).
//  - given != null: a precomputed order (order_kernel) is copied in;
//  - nunits > 0: dimension zones (zone_dims contiguous dimensions) ranked by
//    sum over the zone of (q_j - mu_j)^2 against the block means, best zone
//    first, storage order inside a zone, ties to the lower zone;
//  - otherwise storage order.
__device__ __forceinline__ void put_dim(const WarpSmem &w, int i, int j, const float *__restrict__ qrow,
                                        const float *__restrict__ scale) {
    w.ord[i] = (uint16_t)j;
    if (scale) {
        float sj = scale[j];
        w.qo[i] = qrow[j] / sj;
        w.s2o[i] = sj * sj;
    } else {
        w.qo[i] = qrow[j];
    }
}

__device__ void build_order(const WarpSmem &w, const float *__restrict__ qrow, const float *__restrict__ mu,
                            const uint16_t *__restrict__ given, const float *__restrict__ scale, int d, int zone_dims,
                            int nunits, int lane) {
    if (given) {
        for (int i = lane; i < d; i += 32) put_dim(w, i, given[i], qrow, scale);
        __syncwarp();
        return;
    }
    if (nunits == 0) {
        for (int i = lane; i < d; i += 32) put_dim(w, i, i, qrow, scale);
        __syncwarp();
        return;
    }
    const int Z = zone_dims < 1 ? 1 : zone_dims;
    uint64_t key[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int u = t * 32 + lane;
        key[t] = kEmptyKey;
        if (u < nunits) {
            float sc = 0.f;
            int j1 = min(d, u * Z + Z);
            for (int j = u * Z; j < j1; ++j) {
                float v = qrow[j] - mu[j];
                sc = fmaf(v, v, sc);
            }
            key[t] = ((uint64_t)f2o(-sc) << 32) | (uint32_t)u;
        }
    }
    const int m = (nunits + 31) >> 5;
    if (m <= 1) reg_bitonic_sort<1>(key, lane);
    else if (m <= 2) reg_bitonic_sort<2>(key, lane);
    else if (m <= 4) reg_bitonic_sort<4>(key, lane);
    else reg_bitonic_sort<8>(key, lane);
    // rank r = t*32 + lane holds zone key[t]; rank of the last (shorter) zone
    const int lastlen = d - (nunits - 1) * Z;
    int rlast = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t)
        if (t * 32 + lane < nunits && (int)(key[t] & 0xffffffffu) == nunits - 1) rlast = t * 32 + lane;
    for (int o = 16; o; o >>= 1) rlast = max(rlast, __shfl_xor_sync(kFull, rlast, o));
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int r = t * 32 + lane;
        if (r < nunits) {
            const int z = (int)(key[t] & 0xffffffffu);
            const int off = r * Z - ((r > rlast) ? (Z - lastlen) : 0);
            const int len = (z == nunits - 1) ? lastlen : Z;
            for (int u = 0; u < len; ++u) put_dim(w, off + u, z * Z + u, qrow, scale);
        }
    }
    __syncwarp();
}

// Pruning predicate on a partial distance after `dv` of D dimensions
// (true = discard). `thr` is the slack-widened threshold.
template <int PR>
__device__ __forceinline__ bool prune_test(float partial, float thr, int dv, int D, float eps0, float rx2,
                                           float rq2, float sd2, float bsa_m) {
    if (PR == PR_BOND) {
        return partial > thr;  // Sec. 5: the partial distance is a lower bound
    } else if (PR == PR_ADS) {
        // Sec. 2.3 ADSampling: scaled partial vs tau * (1 + eps0/sqrt(d))^2
        float r = 1.f + eps0 * rsqrtf((float)dv);
        return partial * (float)D > thr * r * r * (float)dv;
    } else if (PR == PR_BSA) {
        // Sec. 2.3 BSA_res on PCA-projected data. Exact part (Cauchy-Schwarz):
        // the unvisited distance is at least (||x_r|| - ||q_r||)^2. Error-
        // quantile part: the visited PCA dimensions hold the fraction
        // frac = F(d) of the collection's variance, so partial / F(d) estimates
        // the full distance; it is tested against tau widened by (1 + m/sqrt(d))^2.
        float g = sqrtf(rx2) - sqrtf(rq2);
        if (partial + g * g > thr) return true;
        float r = 1.f + bsa_m * rsqrtf((float)dv);
        return partial > thr * sd2 * r * r;
    } else if (PR == PR_ADSB) {
        // ADSampling with PDX-BOND's query-aware order: PDX-BOND's exact test,
        // or the hypothesis test against tau scaled by sd2 = F_q(d), the
        // visited share of the vector's expected distance (mass_kernel)
        if (partial > thr) return true;
        float r = 1.f + eps0 * rsqrtf((float)dv);
        return partial > thr * sd2 * r * r;
    } else if (PR == PR_CSIP) {
        // inner product, any norms: partial is the visited sum of q_j x_j and
        // rx2 the Cauchy-Schwarz margin from cs_margin; the unvisited part of
        // -q.x is at least -||q_r|| ||x_r||
        return -partial - rx2 > thr;
    } else {
        return false;
    }
}

// Margin of the Cauchy-Schwarz inner-product bound at a check point: the
// largest value the unvisited dimensions can add to q.x, ||q_r|| ||x_r||, plus
// the rounding of the FP32 sums (the visited partial is within D * 2^-24 of
// sum |q_j x_j| <= ||q|| ||x||; the squared norms are sums of squares with
// the same relative error). rx2, x2: the vector's unvisited and whole squared
// norms; rq2, q2: the query's.
__device__ __forceinline__ float cs_margin(float rx2, float x2, float rq2, float q2, float gamma) {
    return sqrtf(rx2 * rq2) * (1.f + gamma) + gamma * sqrtf(x2 * q2);
}

// Resident CTAs per SM the register allocation is built for (OCC): 3 (80
// registers, 24 warps per SM) or, for FP32 blocks, 4 (64 registers, 32 warps).
// BF16/FP8 blocks stay at 3: their lower-bound arithmetic would spill at 64.
// The launcher takes 4 when four CTAs' shared memory still leaves room for L1.


// Exactness check (finished_log): lane 0 records a vector that passed every
// prune test of the scan and reached the merge with all D dimensions.
__device__ __forceinline__ void log_finished(const ScanParams &a, int64_t qi, int32_t id, int lane) {
    if (lane == 0) {
        const unsigned long long pos = atomicAdd(a.fin_count, 1ull);
        if (pos < a.fin_cap) a.fin_log[pos] = ((uint64_t)qi << 32) | (uint32_t)id;
    }
}

// Offer a full distance to the query's shared pool (lane 0 writes). The pool
// is a ring: once full, new distances (only those below the current
// threshold are offered) replace the oldest. Each (query, vector) pair is
// scanned once, so the pool never holds a vector twice, and the k-th smallest
// of any set of distinct scanned vectors bounds the final k-th from above.
__device__ __forceinline__ void pool_push(const ScanParams &a, int64_t qi, float dist, int lane) {
    if (lane == 0) {
        const unsigned pos = (unsigned)atomicAdd(a.pool_cnt + qi, 1);
        a.pool[qi * kPoolCap + (pos % kPoolCap)] = dist;
    }
}

// k-th smallest distance in the query's pool as an ordered uint32 (+inf when
// fewer than k slots are filled): a bitwise search for the largest key v with
// fewer than k pool keys below it. Slots claimed but not yet written still
// read +inf, which can only raise the result.
__device__ __forceinline__ uint32_t pool_kth(const ScanParams &a, int64_t qi, int k, int lane) {
    const unsigned pushed = (unsigned)*reinterpret_cast<volatile int32_t *>(a.pool_cnt + qi);
    const int n = (int)min(pushed, (unsigned)kPoolCap);
    if (n < k) return 0xff800000u;  // f2o(+inf)
    const volatile float *pl = a.pool + qi * kPoolCap;
    uint32_t v[kPoolCap / 32];
#pragma unroll
    for (int i = 0; i < kPoolCap / 32; ++i) {
        const int idx = lane + 32 * i;
        v[i] = idx < n ? f2o(pl[idx]) : 0xffffffffu;
    }
    uint32_t prefix = 0;
#pragma unroll 1
    for (int bit = 31; bit >= 0; --bit) {
        const uint32_t trial = prefix | (1u << bit);
        int c = 0;
#pragma unroll
        for (int i = 0; i < kPoolCap / 32; ++i) c += v[i] < trial;
        if (__reduce_add_sync(kFull, c) < k) prefix = trial;
    }
    return prefix;
}

// Full distance of one stored vector from its row of the row-major FP32 copy
// (warp-uniform result). With vec4 (d a multiple of 4 and both rows 16-byte
// aligned) lanes take 16-byte pieces i = lane, lane + 32, ... and issue
// kRowUnroll of them (512 bytes per warp each) before the first is consumed;
// otherwise lanes take dimensions j = lane, lane + 32, ... (128 contiguous
// bytes per request). Rounds of 3 (384 dimensions, then the early-exit check
// of row_dist_bounded) beat 2, 4 and 5 (1M x 768: 263k vs 251k / 258k / 251k
// queries/s; 2M x 1536 unchanged).
constexpr int kRowUnroll = 3;
template <int MET>
__device__ __forceinline__ float row_dist(const float *__restrict__ xrow, const float *__restrict__ qrow, int D,
                                          int lane, bool vec4) {
    float acc = 0.f;
    if (vec4) {
        const float4 *x4 = reinterpret_cast<const float4 *>(xrow);
        const float4 *q4 = reinterpret_cast<const float4 *>(qrow);
        const int n4 = D >> 2;
        for (int base = lane; base < n4; base += 32 * kRowUnroll) {
            float4 xv[kRowUnroll];
#pragma unroll
            for (int u = 0; u < kRowUnroll; ++u) {
                const int i = base + 32 * u;
                xv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (i < n4) xv[u] = __ldg(x4 + i);
            }
            // the query row is re-read for every row of the item: an L1 hit
#pragma unroll
            for (int u = 0; u < kRowUnroll; ++u) {
                const int i = base + 32 * u;
                if (i < n4) {
                    const float4 qv = __ldg(q4 + i);
                    acc = term<MET>(qv.x, xv[u].x, acc);
                    acc = term<MET>(qv.y, xv[u].y, acc);
                    acc = term<MET>(qv.z, xv[u].z, acc);
                    acc = term<MET>(qv.w, xv[u].w, acc);
                }
            }
        }
    } else {
        for (int j = lane; j < D; j += 32) acc = term<MET>(qrow[j], __ldg(xrow + j), acc);
    }
    return rank_dist<MET>(warp_sum(acc));
}

// The same with an early exit (L2 / L1, whose partial sums only grow): after
// each round of loads but the last, the partial over the dimensions read so
// far is compared with thr (already slack-widened); above it the vector is
// pruned and *visited < D tells the caller how far it got.
template <int MET>
__device__ __forceinline__ float row_dist_bounded(const float *__restrict__ xrow, const float *__restrict__ qrow,
                                                  int D, int lane, bool vec4, float thr, int *visited) {
    float acc = 0.f;
    *visited = D;
    if (vec4) {
        const float4 *x4 = reinterpret_cast<const float4 *>(xrow);
        const float4 *q4 = reinterpret_cast<const float4 *>(qrow);
        const int n4 = D >> 2;
        for (int base = lane; base < n4; base += 32 * kRowUnroll) {
            float4 xv[kRowUnroll];
#pragma unroll
            for (int u = 0; u < kRowUnroll; ++u) {
                const int i = base + 32 * u;
                xv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (i < n4) xv[u] = __ldg(x4 + i);
            }
#pragma unroll
            for (int u = 0; u < kRowUnroll; ++u) {
                const int i = base + 32 * u;
                if (i < n4) {
                    const float4 qv = __ldg(q4 + i);
                    acc = term<MET>(qv.x, xv[u].x, acc);
                    acc = term<MET>(qv.y, xv[u].y, acc);
                    acc = term<MET>(qv.z, xv[u].z, acc);
                    acc = term<MET>(qv.w, xv[u].w, acc);
                }
            }
            const int done = (base - lane + 32 * kRowUnroll) * 4;  // dimensions read so far
            if (MET != MT_IP && done < D) {
                const float part = warp_sum(acc);
                if (part > thr) {
                    *visited = done;
                    return part;
                }
            }
        }
    } else {
        for (int j0 = 0; j0 < D; j0 += 512) {
            const int j1 = min(D, j0 + 512);
            for (int j = j0 + lane; j < j1; j += 32) acc = term<MET>(qrow[j], __ldg(xrow + j), acc);
            if (MET != MT_IP && j1 < D) {
                const float part = warp_sum(acc);
                if (part > thr) {
                    *visited = j1;
                    return part;
                }
            }
        }
    }
    return rank_dist<MET>(warp_sum(acc));
}

// PRUNE phases with at most this many survivors finish from the row-major
// copy when the index keeps one: at once when every survivor is far below the
// threshold, else once kPruneBudget further dimensions have not pruned them
// (see the kernel). With 8, survivors take one PRUNE step in the visit order
// (8 dimensions after a first step of 4) before the rows (1M x 768: 8 -> 258k
// queries/s, 16 / 32 -> 255k / 250k).
constexpr int kRowFinish = 8;
constexpr int kPruneBudget = 8;

// LOG: the instance that records finished vectors (finished_log); the
// searches' own instances carry none of its code or registers.
template <int PR, int MET, int ST, int OCC, bool LOG = false>
__global__ void __launch_bounds__(256, OCC) pdxsearch_kernel(ScanParams a) {
    using ET = typename Elem<ST>::T;
    constexpr bool kLB = (PR == PR_BOND || PR == PR_NONE);  // low-precision: prune on a lower bound
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int D = a.d;
    const int nunits = sort_units(D, a.zone_dims, a.order, PR, a.qorder != nullptr);
    WarpSmem w = carve(smem + (size_t)warp * warp_smem_bytes(D, a.k, ST == ST_FP8), D, a.k, ST == ST_FP8);
    const ET *xbase = reinterpret_cast<const ET *>(ST == ST_F32 ? static_cast<const void *>(a.data) : a.data_lp);
    const int h = lane >> 4, sl = lane & 15;
    const int k = a.k;
    const int chunks = a.chunks_per_part;
    if (lane < kStats) w.ctr[lane] = 0;
    __syncwarp();

    while (true) {
        unsigned long long wi = 0;
        if (lane == 0) wi = atomicAdd(reinterpret_cast<unsigned long long *>(a.work_counter), 1ull);
        wi = __shfl_sync(kFull, wi, 0);
        if ((int64_t)wi >= a.nitems) break;
        const int slot = a.slot0 + (int)(wi / (unsigned long long)a.nq);
        const int64_t qi = (int64_t)(wi % (unsigned long long)a.nq);
        const int pr = slot / chunks, ch = slot % chunks;
        const int part = a.probes ? a.probes[qi * (a.nslots / chunks) + pr] : a.part0 + pr;
        uint64_t *out = a.cand + ((size_t)qi * a.nslots + slot) * k;
        int b0 = 0, b1 = 0;
        if (part >= 0) {
            b0 = a.part_blk[part] + ch * a.blocks_per_item;
            b1 = min(a.part_blk[part + 1], b0 + a.blocks_per_item);
        }
        if (b0 >= b1) {
            for (int i = lane; i < k; i += 32) out[i] = kEmptyKey;
            continue;
        }
        if (lane == 0) w.ctr[S_ITEMS] += 1;
        const float *qrow = a.q + qi * D;
        // the query as the row-major vectors are stored (untransformed for a
        // rotated or projected index, whose rows keep the original vectors)
        const float *qrow_r = a.qrows + qi * D;
        const uint16_t *given = nullptr;
        if (a.qorder) given = a.qorder + (a.qorder_per_part ? (qi * (a.nslots / chunks) + pr) : qi) * (int64_t)D;
        volatile uint32_t *tau_g_ptr = reinterpret_cast<volatile uint32_t *>(a.tau) + qi;
        // The query's shared τ is read one block ahead: the read a block uses
        // went out with the previous block's loads (the first one before the
        // visit order is built), so a block whose first step is already in
        // registers waits for no load at all. τ only decreases, so a value one
        // block old still bounds the final k-th distance, and the warp's own
        // candidates are in tau_loc.
        // The raw ordered value is kept and converted only when used, so no
        // instruction waits for the read before the next loads go out.
        uint32_t tau_ahead = *tau_g_ptr;
        // Every block of a part but its last holds 64 vectors (parts fill their
        // blocks in order), so only an item's last block reads its count. The
        // item's vectors count as scanned and as pruned up front; blocks take
        // back from the pruned count the vectors that reach the merge.
        const int last_cnt = a.blk_cnt[b1 - 1];
        build_order(w, qrow, a.means ? a.means + (int64_t)part * D : nullptr, given,
                    (ST == ST_FP8) ? a.scale : nullptr, D, a.zone_dims, nunits, lane);
        // every vector takes the first fetch step: its values are counted here,
        // those of later WARMUP steps by the blocks that take them
        const int fs0 = min(D, (PR == PR_NONE) ? D : max(1, a.first_step));
        if (lane == 0) {
            const unsigned long long nv = (unsigned long long)(b1 - b0 - 1) * kBlock + (unsigned)last_cnt;
            w.ctr[S_SCANNED] += nv;
            w.ctr[S_PRUNED] += nv;
            w.ctr[S_VALUES] += nv * (unsigned)fs0;
        }
        int cnt = 0;
        float tau_loc = __int_as_float(0x7f800000);
        const float *qaux = (PR == PR_BSA)    ? a.qaux + qi * a.nchk * 2
                            : (PR == PR_ADSB) ? a.qaux + (qi * (a.nslots / chunks) + pr) * (int64_t)a.nchk
                            : (PR == PR_CSIP) ? a.qaux + qi * (a.nchk + 1) * 2
                                              : nullptr;
        // PDX-BOND skim of the first fetch step (4 dimensions). In exact search
        // nearly every block ends there: each of its vectors' partial over the
        // query's first 4 dimensions already exceeds the threshold. The skim
        // takes two blocks per warp iteration: lanes h = 0 / 1 take blocks sb
        // and sb + 1, lane sl holds vectors 4*sl..4*sl+3 and loads their 4
        // first-step values (one 16-byte load per dimension), so a vector's
        // partial needs no exchange between lanes, and one vote tells whether
        // either block keeps a vector. Only blocks that do enter the generic
        // WARMUP/PRUNE code below, with their first step already in acc (the
        // other block of the pair waits in sk). ADSampling and BSA bounds are
        // loose after 4 dimensions, blocks rarely end there, and those kernels
        // take every block through the generic code.
        const bool skim = (PR == PR_BOND) && a.first_step == 4 && D > 4;
        // The 4 leading dimensions and their query values are re-read from
        // shared memory for every pair rather than held in registers for the
        // item: the 8 registers they would take let the compiler keep more of
        // the generic path's state resident (1M x 768: 229k -> 245k queries/s).
        int sj0 = 0, sj1 = 0, sj2 = 0, sj3 = 0;
        float sq0 = 0.f, sq1 = 0.f, sq2 = 0.f, sq3 = 0.f;
        float ss0 = 1.f, ss1 = 1.f, ss2 = 1.f, ss3 = 1.f;
        int bnext = b0;   // next block the skim (or the plain loop) takes
        int pend = -1;    // block whose skim partials wait in sk (lanes 16..31)
        float4 sk = make_float4(0.f, 0.f, 0.f, 0.f);

        while (true) {
            int b;
            bool first_done = false;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            if (!skim) {
                if (bnext >= b1) break;
                b = bnext++;
            } else {
                if (pend >= 0) {
                    b = pend;
                    pend = -1;
                } else {
                    unsigned vote = 0;
                    int since = 0;
                    while (bnext < b1) {
                        const float thr_s = slack(fminf(tau_loc, o2f(tau_ahead)), a.gamma);
                        // the shared tau moves slowly: re-read every 4th pair
                        if ((++since & 3) == 0) tau_ahead = *tau_g_ptr;
                        const int bb = bnext + h;
                        float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f);
                        unsigned al = 0;
                        if (bb < b1) {
                            const ET *xs = xbase + (int64_t)bb * D * kBlock;
                            {
                                sj0 = w.ord[0] * kBlock + 4 * sl;
                                sj1 = w.ord[1] * kBlock + 4 * sl;
                                sj2 = w.ord[2] * kBlock + 4 * sl;
                                sj3 = w.ord[3] * kBlock + 4 * sl;
                            }
                            const float4 x0 = Elem<ST>::load4(xs + sj0);
                            const float4 x1 = Elem<ST>::load4(xs + sj1);
                            const float4 x2 = Elem<ST>::load4(xs + sj2);
                            const float4 x3 = Elem<ST>::load4(xs + sj3);
                            {
                                sq0 = w.qo[0];
                                sq1 = w.qo[1];
                                sq2 = w.qo[2];
                                sq3 = w.qo[3];
                                if (ST == ST_FP8) {
                                    ss0 = w.s2o[0];
                                    ss1 = w.s2o[1];
                                    ss2 = w.s2o[2];
                                    ss3 = w.s2o[3];
                                }
                            }
                            if (ST == ST_F32) {
                                s4.x = term<MET>(sq3, x3.x, term<MET>(sq2, x2.x, term<MET>(sq1, x1.x, term<MET>(sq0, x0.x, 0.f))));
                                s4.y = term<MET>(sq3, x3.y, term<MET>(sq2, x2.y, term<MET>(sq1, x1.y, term<MET>(sq0, x0.y, 0.f))));
                                s4.z = term<MET>(sq3, x3.z, term<MET>(sq2, x2.z, term<MET>(sq1, x1.z, term<MET>(sq0, x0.z, 0.f))));
                                s4.w = term<MET>(sq3, x3.w, term<MET>(sq2, x2.w, term<MET>(sq1, x1.w, term<MET>(sq0, x0.w, 0.f))));
                            } else {
                                s4.x = lp_term<ST, kLB>(sq3, x3.x, lp_term<ST, kLB>(sq2, x2.x, lp_term<ST, kLB>(sq1, x1.x, lp_term<ST, kLB>(sq0, x0.x, 0.f, ss0), ss1), ss2), ss3);
                                s4.y = lp_term<ST, kLB>(sq3, x3.y, lp_term<ST, kLB>(sq2, x2.y, lp_term<ST, kLB>(sq1, x1.y, lp_term<ST, kLB>(sq0, x0.y, 0.f, ss0), ss1), ss2), ss3);
                                s4.z = lp_term<ST, kLB>(sq3, x3.z, lp_term<ST, kLB>(sq2, x2.z, lp_term<ST, kLB>(sq1, x1.z, lp_term<ST, kLB>(sq0, x0.z, 0.f, ss0), ss1), ss2), ss3);
                                s4.w = lp_term<ST, kLB>(sq3, x3.w, lp_term<ST, kLB>(sq2, x2.w, lp_term<ST, kLB>(sq1, x1.w, lp_term<ST, kLB>(sq0, x0.w, 0.f, ss0), ss1), ss2), ss3);
                            }
                            const int nv = (bb == b1 - 1) ? last_cnt : kBlock;
                            al = (unsigned)(s4.x <= thr_s && 4 * sl < nv) | ((unsigned)(s4.y <= thr_s && 4 * sl + 1 < nv) << 1) |
                                 ((unsigned)(s4.z <= thr_s && 4 * sl + 2 < nv) << 2) |
                                 ((unsigned)(s4.w <= thr_s && 4 * sl + 3 < nv) << 3);
                        }
                        vote = __ballot_sync(kFull, al != 0u);
                        if (vote) {
                            sk = s4;
                            break;
                        }
                        bnext += 2;
                    }
                    if (!vote) break;
                    if (vote & 0xffffu) {
                        b = bnext;
                        if (vote >> 16) pend = bnext + 1;
                    } else {
                        b = bnext + 1;
                    }
                    bnext += 2;
                }
                // this block's first-step partials, in the layout of the generic
                // code (lanes h = 0 hold the sums, lanes h = 1 add zero)
                const bool upper = (b != bnext - 2);  // block sb + 1 of its skim pair
                const int from = upper ? sl + 16 : sl;
                acc.x = __shfl_sync(kFull, sk.x, from);
                acc.y = __shfl_sync(kFull, sk.y, from);
                acc.z = __shfl_sync(kFull, sk.z, from);
                acc.w = __shfl_sync(kFull, sk.w, from);
                if (h) acc = make_float4(0.f, 0.f, 0.f, 0.f);
                first_done = true;
            }
            const ET *xb = xbase + (int64_t)b * D * kBlock;
            const int nvalid = (b == b1 - 1) ? a.blk_cnt[b] : kBlock;
            const float tau_g = o2f(tau_ahead);
            tau_ahead = *tau_g_ptr;
            const float thr = slack(fminf(tau_loc, tau_g), a.gamma);
            unsigned alive = 0xfu;
            if (nvalid < kBlock) {
                alive = 0;
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (4 * sl + c < nvalid) alive |= 1u << c;
            }
            int pos = 0, step = (PR == PR_NONE) ? D : max(1, a.first_step);
            int chk = 0;
            int nsurv = -1;  // -1: still in WARMUP
            float my_p = 0.f;
            int my_v = 0;
            // ---------------- WARMUP ----------------
            while (pos < D) {
                const int e = min(D, pos + step);
                int i = first_done ? e : pos;  // the paired first step is already in acc
                first_done = false;
                for (; i + 8 <= e; i += 8) {
                    float4 x[4];
                    float qv[4], s2[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int ii = i + 2 * u + h;
                        const int j = w.ord[ii];
                        qv[u] = w.qo[ii];
                        s2[u] = (ST == ST_FP8) ? w.s2o[ii] : 1.f;
                        x[u] = Elem<ST>::load4(xb + j * kBlock + 4 * sl);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (ST == ST_F32) {
                            acc.x = term<MET>(qv[u], x[u].x, acc.x);
                            acc.y = term<MET>(qv[u], x[u].y, acc.y);
                            acc.z = term<MET>(qv[u], x[u].z, acc.z);
                            acc.w = term<MET>(qv[u], x[u].w, acc.w);
                        } else {
                            acc.x = lp_term<ST, kLB>(qv[u], x[u].x, acc.x, s2[u]);
                            acc.y = lp_term<ST, kLB>(qv[u], x[u].y, acc.y, s2[u]);
                            acc.z = lp_term<ST, kLB>(qv[u], x[u].z, acc.z, s2[u]);
                            acc.w = lp_term<ST, kLB>(qv[u], x[u].w, acc.w, s2[u]);
                        }
                    }
                }
                // the remaining (< 8) dimensions: up to 4 pairs, every load
                // issued before the first is consumed (one round trip)
                if (i < e) {
                    float4 x[4];
                    float qv[4], s2[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int ii = i + 2 * u + h;
                        qv[u] = 0.f;
                        s2[u] = 1.f;
                        x[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (ii < e) {
                            const int j = w.ord[ii];
                            qv[u] = w.qo[ii];
                            if (ST == ST_FP8) s2[u] = w.s2o[ii];
                            x[u] = Elem<ST>::load4(xb + j * kBlock + 4 * sl);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (i + 2 * u + h < e) {
                            if (ST == ST_F32) {
                                acc.x = term<MET>(qv[u], x[u].x, acc.x);
                                acc.y = term<MET>(qv[u], x[u].y, acc.y);
                                acc.z = term<MET>(qv[u], x[u].z, acc.z);
                                acc.w = term<MET>(qv[u], x[u].w, acc.w);
                            } else {
                                acc.x = lp_term<ST, kLB>(qv[u], x[u].x, acc.x, s2[u]);
                                acc.y = lp_term<ST, kLB>(qv[u], x[u].y, acc.y, s2[u]);
                                acc.z = lp_term<ST, kLB>(qv[u], x[u].z, acc.z, s2[u]);
                                acc.w = lp_term<ST, kLB>(qv[u], x[u].w, acc.w, s2[u]);
                            }
                        }
                    }
                }
                pos = e;
                step <<= 1;
                if (PR == PR_NONE || pos >= D) break;
                // predicate on all vectors of the block
                const float4 f = make_float4(acc.x + __shfl_xor_sync(kFull, acc.x, 16),
                                             acc.y + __shfl_xor_sync(kFull, acc.y, 16),
                                             acc.z + __shfl_xor_sync(kFull, acc.z, 16),
                                             acc.w + __shfl_xor_sync(kFull, acc.w, 16));
                float rq2 = 0.f, sd2 = 0.f;
                if (PR == PR_BSA) {
                    rq2 = qaux[chk * 2];
                    sd2 = qaux[chk * 2 + 1];
                }
                if (PR == PR_ADSB) sd2 = qaux[min(chk, a.nchk - 1)];
                if (PR == PR_CSIP) {  // the query's unvisited and whole squared norms
                    rq2 = qaux[(chk + 1) * 2];
                    sd2 = qaux[0];
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    float rx2 = 0.f;
                    if (PR == PR_BSA) rx2 = a.resid[((int64_t)b * a.nchk + chk) * kBlock + 4 * sl + c];
                    if (PR == PR_CSIP) {
                        const float *rb = a.resid + (int64_t)b * (a.nchk + 1) * kBlock + 4 * sl + c;
                        rx2 = cs_margin(rb[(chk + 1) * kBlock], rb[0], rq2, sd2, a.gamma);
                    }
                    if (prune_test<PR>(sel4(f, c), thr, pos, D, a.eps0, rx2, rq2, sd2, a.bsa_m)) alive &= ~(1u << c);
                }
                ++chk;
                if (!__any_sync(kFull, alive != 0u)) {
                    nsurv = 0;
                    break;
                }
                unsigned m0 = __ballot_sync(kFull, alive & 1u) & 0xffffu;
                unsigned m1 = __ballot_sync(kFull, alive & 2u) & 0xffffu;
                unsigned m2 = __ballot_sync(kFull, alive & 4u) & 0xffffu;
                unsigned m3 = __ballot_sync(kFull, alive & 8u) & 0xffffu;
                int nalive = __popc(m0) + __popc(m1) + __popc(m2) + __popc(m3);
                if (nalive <= a.sel_count) {
                    // PRUNE: positions array of the survivors, in slot order
                    unsigned below = (1u << sl) - 1u;
                    int before = __popc(m0 & below) + __popc(m1 & below) + __popc(m2 & below) + __popc(m3 & below);
                    if (h == 0) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            if (alive & (1u << c)) {
                                w.sv[before] = 4 * sl + c;
                                w.sp[before] = sel4(f, c);
                                ++before;
                            }
                        }
                    }
                    __syncwarp();
                    nsurv = nalive;
                    if (lane == 0) w.ctr[S_PBLOCKS] += 1;
                    break;
                }
            }
            // values of the WARMUP steps after the first: dimensions fs0..pos of every vector
            if (pos > fs0 && lane == 0) w.ctr[S_VALUES] += (unsigned long long)(pos - fs0) * nvalid;
            // ---------------- PRUNE ----------------
            // A few survivors: in the dimension-major block every remaining value
            // of one vector sits in its own 256-byte slice, one memory sector per
            // 4-byte value. With a row-major FP32 copy of the vectors their exact
            // distances are finished from contiguous rows instead (D / 32 coalesced
            // 128-byte requests per vector); the merge below takes them as full
            // distances, as it does after the last PRUNE step.
            // Only survivors still far below the threshold (partial < thr / 2 after
            // the dimensions visited so far, e.g. cluster-mates of the query,
            // which need nearly all dimensions) go to the rows; a block with a
            // survivor near the threshold keeps the PRUNE phase, whose visit
            // order prunes such vectors within a few more dimensions.
            bool rows = false;
            if (nsurv > 0 && nsurv <= kRowFinish && a.xnary != nullptr) {
                float spmax = 0.f;
                for (int m = 0; m < nsurv; ++m) spmax = fmaxf(spmax, w.sp[m]);
                rows = __shfl_sync(kFull, (int)(spmax < 0.5f * thr), 0) != 0;
            }
            // Otherwise survivor m owns G = 32 / pow2(nsurv) consecutive lanes; its lanes
            // stride over the step's dimensions, so all lanes stay busy for any
            // mix of survivor count and step size, and a log2(G) shuffle tree
            // reduces each survivor's step sum.
            if (nsurv > 0 && !rows) {
                const int prune_pos0 = pos;
                int G = 32 / pow2_ceil(nsurv);
                int m = lane / G, g = lane % G;
                if (m < nsurv) {
                    my_v = w.sv[m];
                    my_p = w.sp[m];
                }
                __syncwarp();
                while (pos < D) {
                    const int e = min(D, pos + step);
                    float acc1 = 0.f;
                    if (m < nsurv) {
                        // 4 of this lane's dimensions per round: all loads
                        // issued before the first is consumed
                        for (int i = pos + g; i < e; i += 4 * G) {
                            float xv[4], qv[4], s2[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int ii = i + u * G;
                                xv[u] = 0.f;
                                qv[u] = 0.f;
                                s2[u] = 1.f;
                                if (ii < e) {
                                    xv[u] = Elem<ST>::load1(xb + (int)w.ord[ii] * kBlock + my_v);
                                    qv[u] = w.qo[ii];
                                    if (ST == ST_FP8) s2[u] = w.s2o[ii];
                                }
                            }
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                if (i + u * G < e) {
                                    if (ST == ST_F32)
                                        acc1 = term<MET>(qv[u], xv[u], acc1);
                                    else
                                        acc1 = lp_term<ST, kLB>(qv[u], xv[u], acc1, s2[u]);
                                }
                            }
                        }
                    }
                    for (int o = G >> 1; o; o >>= 1) acc1 += __shfl_xor_sync(kFull, acc1, o);
                    my_p += acc1;
                    if (lane == 0) w.ctr[S_VALUES] += (unsigned long long)(e - pos) * nsurv;
                    pos = e;
                    step <<= 1;
                    if (pos >= D) break;
                    float rx2 = 0.f, rq2 = 0.f, sd2 = 0.f;
                    if (PR == PR_BSA) {
                        rq2 = qaux[chk * 2];
                        sd2 = qaux[chk * 2 + 1];
                        if (m < nsurv) rx2 = a.resid[((int64_t)b * a.nchk + chk) * kBlock + my_v];
                    }
                    if (PR == PR_ADSB) sd2 = qaux[min(chk, a.nchk - 1)];
                    if (PR == PR_CSIP && m < nsurv) {
                        const float *rb = a.resid + (int64_t)b * (a.nchk + 1) * kBlock + my_v;
                        rx2 = cs_margin(rb[(chk + 1) * kBlock], rb[0], qaux[(chk + 1) * 2], qaux[0], a.gamma);
                    }
                    ++chk;
                    bool keep = (m < nsurv) && !prune_test<PR>(my_p, thr, pos, D, a.eps0, rx2, rq2, sd2, a.bsa_m);
                    unsigned km = __ballot_sync(kFull, keep && g == 0);   // one bit per survivor, at its lane m*G
                    int nn = __popc(km);
                    if (nn < nsurv) {
                        nsurv = nn;
                        if (nn == 0) break;
                        int Gn = 32 / pow2_ceil(nn);
                        int mn = lane / Gn;
                        unsigned mm = km;
                        for (int t = 0; t < mn && t < nn; ++t) mm &= mm - 1u;
                        int src = (mn < nn) ? (__ffs(mm) - 1) : lane;
                        float np = __shfl_sync(kFull, my_p, src);
                        int nv = __shfl_sync(kFull, my_v, src);
                        if (mn < nn) {
                            my_p = np;
                            my_v = nv;
                        }
                        G = Gn;
                        m = mn;
                        g = lane % Gn;
                    }
                    // survivors that kPruneBudget more dimensions did not prune
                    // need most of the remaining ones: finish them from the rows
                    if (a.xnary != nullptr && nsurv <= kRowFinish && pos - prune_pos0 >= kPruneBudget) {
                        rows = true;
                        break;
                    }
                }
                // survivors' leaders hold (my_v, my_p) at lanes m*G; gather them
                // to lanes 0..nsurv-1 for the merge below
                if (nsurv > 0) {
                    int src = lane * G;
                    float np = __shfl_sync(kFull, my_p, src & 31);
                    int nv = __shfl_sync(kFull, my_v, src & 31);
                    my_p = np;
                    my_v = nv;
                    if (rows) {
                        if (lane < nsurv) w.sv[lane] = my_v;
                        __syncwarp();
                    }
                }
            }
            // ---------------- merge ----------------
            // Candidates are tested against this block's threshold thr (its
            // shared part read one block ahead): tau only decreases, so a
            // distance above thr cannot be among the final k, and one below
            // it that the current tau would reject costs a list entry only.
            // No test waits for a fresh read of the shared tau.
            int nfinal = 0;
            bool pushed = false;
            if (nsurv < 0) {
                // finished in WARMUP: every alive vector has its full distance
                const float4 fm = make_float4(acc.x + __shfl_xor_sync(kFull, acc.x, 16),
                                              acc.y + __shfl_xor_sync(kFull, acc.y, 16),
                                              acc.z + __shfl_xor_sync(kFull, acc.z, 16),
                                              acc.w + __shfl_xor_sync(kFull, acc.w, 16));
                for (int c = 0; c < 4; ++c) {
                    float dist = rank_dist<MET>(sel4(fm, c));
                    bool cand = (h == 0) && (alive & (1u << c)) && (dist <= thr);
                    unsigned cm = __ballot_sync(kFull, cand);
                    while (cm) {
                        int src = __ffs(cm) - 1;
                        cm &= cm - 1u;
                        float dd = __shfl_sync(kFull, dist, src);
                        int v = 4 * src + c;
                        const int id = a.ids[(int64_t)b * kBlock + v];
                        if (ST != ST_F32) dd = row_dist<MT_L2>(a.xnary + (int64_t)id * D, qrow_r, D, lane, a.rows_vec4);  // exact FP32
                        uint64_t key = make_key(dd, id);
                        topk_insert(w.topk, cnt, k, key, lane);
                        if (lane == 0) w.ctr[S_CAND] += 1;
                        // lane 0 reads the shared threshold and the warp follows it
                        if (a.pool && dd < thr) {
                            pool_push(a, qi, dd, lane);
                            pushed = true;
                        }
                    }
                }
                unsigned m0 = __ballot_sync(kFull, alive & 1u) & 0xffffu;
                unsigned m1 = __ballot_sync(kFull, alive & 2u) & 0xffffu;
                unsigned m2 = __ballot_sync(kFull, alive & 4u) & 0xffffu;
                unsigned m3 = __ballot_sync(kFull, alive & 8u) & 0xffffu;
                nfinal = __popc(m0) + __popc(m1) + __popc(m2) + __popc(m3);
                if (LOG) {  // every alive vector: lane l of the first half holds 4l..4l+3
                    const unsigned mm[4] = {m0, m1, m2, m3};
                    for (int c = 0; c < 4; ++c)
                        for (unsigned am = mm[c]; am; am &= am - 1u)
                            log_finished(a, qi, a.ids[(int64_t)b * kBlock + 4 * (__ffs(am) - 1) + c], lane);
                }
            } else if (rows) {
                int finished = 0;
                // all survivors' ids in one round of loads (lane m: survivor m)
                const int myid = (lane < nsurv) ? a.ids[(int64_t)b * kBlock + w.sv[lane]] : 0;
                for (int m = 0; m < nsurv; ++m) {
                    const int id = __shfl_sync(kFull, myid, m);
                    // the row is read in rounds; a partial above the block's
                    // threshold ends it early (the vector is pruned)
                    int vis;
                    const float dd = row_dist_bounded<MET>(a.xnary + (int64_t)id * D, qrow_r, D, lane, a.rows_vec4,
                                                           thr, &vis);
                    if (lane == 0) w.ctr[S_VALUES] += (unsigned long long)vis;
                    if (vis < D) continue;
                    ++finished;
                    if (LOG) log_finished(a, qi, id, lane);
                    if (dd <= thr) {
                        topk_insert(w.topk, cnt, k, make_key(dd, id), lane);
                        if (lane == 0) w.ctr[S_CAND] += 1;
                        if (a.pool && dd < thr) {
                            pool_push(a, qi, dd, lane);
                            pushed = true;
                        }
                    }
                }
                nfinal = finished;
            } else if (nsurv > 0) {
                if (LOG) {
                    const int myid = (lane < nsurv) ? a.ids[(int64_t)b * kBlock + my_v] : 0;
                    for (int m = 0; m < nsurv; ++m) log_finished(a, qi, __shfl_sync(kFull, myid, m), lane);
                }
                float dist = rank_dist<MET>(my_p);
                bool cand = (lane < nsurv) && (dist <= thr);
                unsigned cm = __ballot_sync(kFull, cand);
                while (cm) {
                    int src = __ffs(cm) - 1;
                    cm &= cm - 1u;
                    float dd = __shfl_sync(kFull, dist, src);
                    int v = __shfl_sync(kFull, my_v, src);
                    const int id = a.ids[(int64_t)b * kBlock + v];
                    if (ST != ST_F32) dd = row_dist<MT_L2>(a.xnary + (int64_t)id * D, qrow_r, D, lane, a.rows_vec4);  // exact FP32
                    uint64_t key = make_key(dd, id);
                    topk_insert(w.topk, cnt, k, key, lane);
                    if (lane == 0) w.ctr[S_CAND] += 1;
                    if (a.pool && dd < thr) {
                        pool_push(a, qi, dd, lane);
                        pushed = true;
                    }
                }
                nfinal = nsurv;
            }
            if (nfinal > 0 && lane == 0) w.ctr[S_PRUNED] -= (unsigned long long)nfinal;
            if (nfinal > 0 && cnt == k && !a.tau_fixed) {  // the list changes only through vectors that reach the merge
                float t = key_dist(w.topk[k - 1]);
                if (t < tau_loc) {
                    tau_loc = t;
                    if (lane == 0 && f2o(t) < *tau_g_ptr) atomicMin(reinterpret_cast<unsigned *>(a.tau) + qi, f2o(t));
                }
            }
            if (pushed) {
                // the k-th best over all warps' finds so far
                const uint32_t kt = pool_kth(a, qi, k, lane);
                if (lane == 0 && kt < *tau_g_ptr) atomicMin(reinterpret_cast<unsigned *>(a.tau) + qi, kt);
            }
        }
        for (int i = lane; i < k; i += 32) out[i] = (i < cnt) ? w.topk[i] : kEmptyKey;
        __syncwarp();
    }
    __syncwarp();
    if (lane == 0 && a.counters) {
        atomicAdd(a.counters + C_VALUES, w.ctr[S_VALUES]);
        atomicAdd(a.counters + C_SCANNED, w.ctr[S_SCANNED]);
        atomicAdd(a.counters + C_PRUNED, w.ctr[S_PRUNED]);
        atomicAdd(a.counters + C_PRUNE_BLOCKS, w.ctr[S_PBLOCKS]);
        atomicAdd(a.counters + C_CANDIDATES, w.ctr[S_CAND]);
        atomicAdd(a.counters + C_ITEMS, w.ctr[S_ITEMS]);
    }
}

template <int PR, int MET, int ST>
static cudaError_t launch_scan_t(const ScanParams &p, int num_sms, cudaStream_t st) {
    const int nunits = sort_units(p.d, p.zone_dims, p.order, PR, p.qorder != nullptr);
    if (nunits > kMaxSortUnits) return cudaErrorInvalidValue;
    const size_t per_warp = warp_smem_bytes(p.d, p.k, ST == ST_FP8);
    int warps = 8;
    while (warps > 1 && per_warp * warps > 200 * 1024) warps >>= 1;
    const size_t smem = per_warp * warps;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    // 4 resident CTAs (the 64-register build) when four CTAs' shared memory
    // leaves at least 32 KB of the SM for L1
    const bool four = p.ctas_per_sm != 3 && 4 * (smem + 1024) + 32 * 1024 <= 228 * 1024;
    auto kern = four ? pdxsearch_kernel<PR, MET, ST, 4> : pdxsearch_kernel<PR, MET, ST, 3>;
    if constexpr (ST == ST_F32 && (PR == PR_BOND || PR == PR_CSIP)) {
        if (p.fin_log) kern = four ? pdxsearch_kernel<PR, MET, ST, 4, true> : pdxsearch_kernel<PR, MET, ST, 3, true>;
    } else {
        if (p.fin_log) return cudaErrorInvalidValue;  // the log exists for FP32 BOND and CS_IP scans
    }
    cudaError_t e = raise_smem_limit(kern, smem);
    if (e != cudaSuccess) return e;
    // Shared-memory carveout sized for the requested number of resident CTAs
    // (1 KB reserved per CTA); what remains of the SM's on-chip memory is L1,
    // which holds the lines of the scan's loads in flight.
    const int want = p.ctas_per_sm > 0 ? (int)p.ctas_per_sm : (four ? 4 : 3);
    int pct = (int)((want * (smem + 1024) * 100 + 228 * 1024 - 1) / (228 * 1024));
    if (pct > 100) pct = 100;
    if (pct < 1) pct = 1;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (per_sm > want) per_sm = want;
    int64_t grid = (int64_t)num_sms * per_sm;
    int64_t need = (p.nitems + warps - 1) / warps;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, warps * 32, smem, st>>>(p);
    return counted(cudaGetLastError());
}

template <int ST>
static cudaError_t launch_scan_lp(int pruner, const ScanParams &p, int num_sms, cudaStream_t st) {
    switch (pruner) {
    case PR_NONE: return launch_scan_t<PR_NONE, MT_L2, ST>(p, num_sms, st);
    case PR_BOND: return launch_scan_t<PR_BOND, MT_L2, ST>(p, num_sms, st);
    case PR_ADS: return launch_scan_t<PR_ADS, MT_L2, ST>(p, num_sms, st);
    case PR_BSA: return launch_scan_t<PR_BSA, MT_L2, ST>(p, num_sms, st);
    case PR_ADSB: return launch_scan_t<PR_ADSB, MT_L2, ST>(p, num_sms, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_scan(int pruner, int metric, const ScanParams &p, int num_sms, cudaStream_t st) {
    if (p.nitems == 0) return cudaSuccess;
    if (p.storage != ST_F32) {
        // low-precision storage: L2 only (lower bound / FP32 rerank are L2)
        if (metric != MT_L2) return cudaErrorInvalidValue;
        return p.storage == ST_BF16 ? launch_scan_lp<ST_BF16>(pruner, p, num_sms, st)
                                    : launch_scan_lp<ST_FP8>(pruner, p, num_sms, st);
    }
    switch (pruner) {
    case PR_NONE:
        if (metric == MT_IP) return launch_scan_t<PR_NONE, MT_IP, ST_F32>(p, num_sms, st);
        if (metric == MT_L1) return launch_scan_t<PR_NONE, MT_L1, ST_F32>(p, num_sms, st);
        return launch_scan_t<PR_NONE, MT_L2, ST_F32>(p, num_sms, st);
    case PR_BOND:
        if (metric == MT_L1) return launch_scan_t<PR_BOND, MT_L1, ST_F32>(p, num_sms, st);
        return launch_scan_t<PR_BOND, MT_L2, ST_F32>(p, num_sms, st);
    case PR_ADS:
        return launch_scan_t<PR_ADS, MT_L2, ST_F32>(p, num_sms, st);
    case PR_BSA:
        return launch_scan_t<PR_BSA, MT_L2, ST_F32>(p, num_sms, st);
    case PR_ADSB:
        return launch_scan_t<PR_ADSB, MT_L2, ST_F32>(p, num_sms, st);
    case PR_CSIP:
        if (metric != MT_IP) return cudaErrorInvalidValue;
        return launch_scan_t<PR_CSIP, MT_IP, ST_F32>(p, num_sms, st);
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace pdx
