// Dense (unpruned) exact k-NN on the 5th-generation tensor cores.
//
// Without pruning every query meets every vector, and the L2 distance splits
// into ||q||^2 + ||x||^2 - 2 q.x (Sec. 2.1): the only term that couples q and
// x is one entry of the product Q X^T, a dense contraction over the D
// dimensions. This file computes that product tile by tile on tcgen05 and
// turns it into exact top-k results:
//
//   1. prep      copy the queries into an aligned buffer, ||q|| per query,
//                reset the per-query state.
//   2. gemm      persistent, warp-specialised: one thread issues TMA loads of
//                128x32 query and 256x32 vector FP32 tiles (128-byte swizzle)
//                into a 4-stage shared-memory ring, one thread issues
//                tcgen05.mma kind::tf32 (M=128, N=256, K=8) into one of two
//                TMEM accumulators, 8 or 16 epilogue warps drain the other
//                accumulator with tcgen05.ld. For every (query, vector) the epilogue forms
//                est = ||x||^2 - 2 acc (L2) or -acc (IP) and a proven error
//                margin m (TF32 operands, FP32 accumulation; see dense_bounds),
//                so that est - m <= exact <= est + m. The kernel runs twice.
//                In the bound pass each epilogue thread keeps the k smallest
//                upper bounds of its query over all the tiles its CTA serves
//                for that query tile (a run; the grid is a multiple of the
//                query tiles, so one run per CTA) and appends them at the
//                end. The emit pass lists the vectors whose lower bound is
//                within T*.
//   3. select    one CTA per query: T* = k-th smallest of those upper bounds,
//                which is the k-th smallest upper bound over all vectors.
//   4. finish    one CTA per query: every listed vector gets its exact FP32
//                distance (same lanes and reduction as the scan path's
//                refine), and the k best (distance, id) keys are kept.
//
// Why this is exact: the true k nearest have lower <= exact <= k-th exact
// distance <= T* (T* is the k-th of upper bounds, each above its own exact
// distance), so they are listed; the FP32 rerank decides among the listed.
// A threshold shared between tiles while the GEMM runs cannot work here: a
// tile of random vectors rarely holds k near neighbours of a query, so its
// local k-th stays at the far distances (clustered data), and the list would
// hold a large part of the collection. Two passes cost a second GEMM and give
// the smallest candidate list the margin allows.
// If a query lists more vectors than its buffer holds, or the GEMM gave up on
// a wait, the finish kernel computes that query's result by a plain FP32 scan
// of all vectors instead (counted in the search statistics).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <mutex>

#include "pdx_internal.cuh"

namespace pdx {
namespace {

constexpr int TM = 128;                 // queries per tile = TMEM lanes
constexpr int TN = 256;                 // vectors per tile = accumulator columns
constexpr int TKF = 32;                 // FP32 elements per K chunk = one 128-byte swizzle row
constexpr int STAGES = 4;
constexpr int A_BYTES = TM * TKF * 4;   // 16 KB
constexpr int B_BYTES = TN * TKF * 4;   // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
// Epilogue warps: EW per TMEM lane quarter, each draining TN / EW columns
// (EW = 4 for k <= 16, 2 for the larger register lists of k <= 64).
template <int EW> struct Epi {
    static constexpr int warps = 4 * EW;
    static constexpr int threads = (2 + warps) * 32;
    static constexpr int span = TN / EW;
};
constexpr int ew_for(int k) { return k <= 16 ? 4 : 2; }
constexpr int TMEM_COLS = 2 * TN;       // two accumulators
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;  // + alignment of the swizzled tiles
constexpr uint64_t kWaitNs = 2000000000ull;              // give up on a barrier after 2 s

// Instruction descriptor of tcgen05.mma kind::tf32: FP32 accumulator (bits
// 4-5 = 1), A and B TF32 (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 =
// 0), N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bounded wait for the phase of the given parity. Gives up after kWaitNs, or
// as soon as another role of the CTA has given up, and reports it.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer() - t0 > kWaitNs) {
            *abort_flag = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// rows of 128 bytes, groups of 8 rows 1024 bytes apart (stride byte offset),
// descriptor version 1 at bit 46, swizzle mode 2 (128 B) at bits 61-63. The
// leading byte offset is not used by this layout.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct DenseParams {
    int64_t nq, n;
    int32_t d, k;
    int32_t nqt;                 // query tiles
    int64_t ntiles;              // query tiles x vector tiles
    const float2 *qnorm;         // [nq] (||tf32(q)||, ||q - tf32(q)||), rounded up
    const float4 *xnorm;         // [n] (||x||^2, ||x||, ||x - tf32(x)||, 0), norms rounded up
    float *ubuf;                 // bound pass: [nq][ucap] the k smallest upper bounds of each
                                 // (CTA, row, column part) run, appended
    int32_t *ucnt;               // [nq] values appended
    int32_t ucap;
    const float *tstar;          // emit pass: [nq] k-th smallest upper bound over all vectors
    int32_t *cnt;                // [nq] entries emitted
    int32_t cap;                 // entries per query
    int32_t *ent_id;             // [nq][cap] emitted vector ids
    float k2, c_acc, c_xx, c_rel;  // margin coefficients (see dense_bounds)
    int32_t *err;                // set when a wait gave up
    int32_t stall_test;          // test hook: the producer issues no loads, so the
                                 // first wait of the MMA thread runs out
};

// Error margin of est for one (query, vector) pair. Both operands are
// rounded to TF32 before the GEMM (q~, x~), so the tensor core's own
// conversion is exact, and TF32 x TF32 products are exact in FP32. Then
//   q.x - q~.x~ = (q - q~).x + q~.(x - x~),
// so |q.x - q~.x~| <= ||q - q~|| ||x|| + ||q~|| ||x - x~|| (Cauchy-Schwarz, with
// the residual norms measured per row), and FP32 accumulation of the D exact
// products adds at most c_acc sum_j |q~_j x~_j| <= c_acc ||q~|| ||x~||, with
// ||x~|| <= ||x|| + ||x - x~||. For L2 the dot enters twice (k2 = 2); ||x||^2
// carries its FP32 rounding (c_xx) and forming est rounds once more (c_rel).
// Per row: P = k2 ||q~|| (1 + c_acc), Q = k2 (||q - q~|| + c_acc ||q~||), and
//   m = P ||x - x~|| + Q ||x|| + c_xx ||x||^2 + c_rel |est|.
template <int MET>
__device__ __forceinline__ void dense_bounds(float acc, float4 xn, float P, float Q, const DenseParams &p, float &lo,
                                             float &up) {
    float est, m;
    if (MET == MT_L2) {
        est = fmaf(-2.f, acc, xn.x);
        m = fmaf(P, xn.z, fmaf(Q, xn.y, fmaf(p.c_xx, xn.x, p.c_rel * fabsf(est))));
    } else {
        est = -acc;
        m = fmaf(P, xn.z, fmaf(Q, xn.y, p.c_rel * fabsf(est)));
    }
    lo = est - m;
    up = est + m;
}

template <int KL, int MET, int MODE, int EW>
__global__ void __launch_bounds__(Epi<EW>::threads, 1)
    dense_tc_kernel(const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmX, DenseParams p) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[2 * STAGES + 5];
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // barriers: full[s], empty[s], tfull[b], tempty[b], done
    auto full = [&](int s) { return smem_u32(&bars[s]); };
    auto empty = [&](int s) { return smem_u32(&bars[STAGES + s]); };
    auto tfull = [&](int b) { return smem_u32(&bars[2 * STAGES + b]); };
    auto tempty = [&](int b) { return smem_u32(&bars[2 * STAGES + 2 + b]); };
    const uint32_t done = smem_u32(&bars[2 * STAGES + 4]);
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull(b), 1);
            mbar_init(tempty(b), Epi<EW>::warps);
        }
        mbar_init(done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_holder;
    const int nk = (p.d + TKF - 1) / TKF;
    volatile int *ab = &abort_flag;

    if (warp == 0) {
        // ---- TMA producer ----
        if (lane == 0 && !p.stall_test) {
            int s = 0;
            uint32_t ph = 0;
            uint32_t issued = 0, last_par = 0;  // per stage: loads issued, parity of the last one
            for (int64_t t = blockIdx.x; t < p.ntiles && !*ab; t += gridDim.x) {
                const int qt = (int)(t % p.nqt);
                const int nt = (int)(t / p.nqt);
                for (int kc = 0; kc < nk; ++kc) {
                    if (!wait_bar(empty(s), ph ^ 1u, ab)) break;
                    const uint32_t a = sbase + s * STAGE_BYTES, b = a + A_BYTES;
                    mbar_expect_tx(full(s), STAGE_BYTES);
                    tma_load_2d(a, &tmQ, full(s), kc * TKF, qt * TM);
                    tma_load_2d(b, &tmX, full(s), kc * TKF, nt * TN);
                    issued |= 1u << s;
                    last_par = (last_par & ~(1u << s)) | (ph << s);
                    if (++s == STAGES) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (*ab) {
                // copies in flight must land before the CTA's shared memory goes away
                int dummy = 0;
                for (int st = 0; st < STAGES; ++st)
                    if (issued & (1u << st)) wait_bar(full(st), (last_par >> st) & 1u, &dummy);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int it = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x, ++it) {
                const int b = it & 1;
                const uint32_t use = (uint32_t)(it >> 1);
                if (!wait_bar(tempty(b), (use & 1u) ^ 1u, ab)) break;
                tc_fence_after();
                const uint32_t dt = tbase + (uint32_t)(b * TN);
                for (int kc = 0; kc < nk; ++kc) {
                    if (!wait_bar(full(s), ph, ab)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a = sbase + s * STAGE_BYTES;
                    const uint64_t ad = sw128_desc(a), bd = sw128_desc(a + A_BYTES);
#pragma unroll
                    for (int kk = 0; kk < TKF / 8; ++kk)  // K = 8 TF32 = 32 bytes per instruction
                        mma_tf32(dt, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), (kc | kk) != 0);
                    mma_commit(empty(s));  // the stage is free once these MMAs have read it
                    if (++s == STAGES) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (ok) mma_commit(tfull(b));
            }
            // no MMA may be in flight when TMEM is released
            mma_commit(done);
            int dummy = 0;
            wait_bar(done, 0, &dummy);
        }
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32*(w%4).. (its quarter) and
        // columns [part*span, (part+1)*span) with part = (w-2)/4 ----
        constexpr int SPAN = Epi<EW>::span;
        const int quarter = warp & 3;
        const int part = (warp - 2) >> 2;
        const int row_in_tile = quarter * 32 + lane;
        // bound pass: the k smallest upper bounds of this thread's row over all
        // its tiles of one query tile (a run), appended when the run ends
        float L[KL];
#pragma unroll
        for (int i = 0; i < KL; ++i) L[i] = __int_as_float(0x7f800000);
        int64_t run_row = -1;
        auto flush = [&]() {
            if (MODE == 0 && run_row >= 0 && run_row < p.nq) {
                int nf = 0;
#pragma unroll
                for (int i = 0; i < KL; ++i) nf += (i < p.k && L[i] < __int_as_float(0x7f800000)) ? 1 : 0;
                if (nf > 0) {
                    const int pos = atomicAdd(p.ucnt + run_row, nf);
                    float *u = p.ubuf + run_row * p.ucap;
#pragma unroll
                    for (int i = 0; i < KL; ++i)
                        if (i < nf && pos + i < p.ucap) u[pos + i] = L[i];
                }
            }
#pragma unroll
            for (int i = 0; i < KL; ++i) L[i] = __int_as_float(0x7f800000);
        };
        int it = 0;
        for (int64_t t = blockIdx.x; t < p.ntiles; t += gridDim.x, ++it) {
            const int b = it & 1;
            const uint32_t use = (uint32_t)(it >> 1);
            const int qt = (int)(t % p.nqt);
            const int64_t nt = t / p.nqt;
            // one lane waits and the warp follows its verdict, so that the
            // warp-collective TMEM loads below never run with lanes missing
            int ok = 1;
            if (lane == 0) ok = wait_bar(tfull(b), use & 1u, ab) ? 1 : 0;
            if (!__shfl_sync(kFull, ok, 0)) break;
            tc_fence_after();
            const int64_t r = (int64_t)qt * TM + row_in_tile;
            const bool rv = r < p.nq;
            if (MODE == 0 && r != run_row) {
                flush();
                run_row = r;
            }
            float P = 0.f, Q = 0.f;
            if (rv) {
                const float2 qn = __ldg(p.qnorm + r);
                P = p.k2 * qn.x * (1.f + p.c_acc);
                Q = p.k2 * (qn.y + p.c_acc * qn.x);
            }
            const int64_t col0 = nt * TN + part * SPAN;
            const uint32_t taddr = tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * TN + part * SPAN);
            const float T = (MODE == 1 && rv) ? __ldg(p.tstar + r) : __int_as_float(0xff800000);
#pragma unroll 1
            for (int cb = 0; cb < SPAN; cb += 32) {
                // the chunk's per-vector norms: one coalesced load, then each
                // column's values are broadcast to the warp by shuffles
                const int64_t cbase = col0 + cb;
                const int64_t left = p.n - cbase;
                const int nvalid = left <= 0 ? 0 : (left >= 32 ? 32 : (int)left);
                const float4 mine = lane < nvalid ? __ldg(p.xnorm + cbase + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
                float v[32];
                tmem_ld32(taddr + cb, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float4 xn = make_float4(__shfl_sync(kFull, mine.x, i), __shfl_sync(kFull, mine.y, i),
                                                  __shfl_sync(kFull, mine.z, i), 0.f);
                    if (rv && i < nvalid) {
                        float lo, up;
                        dense_bounds<MET>(v[i], xn, P, Q, p, lo, up);
                        if (MODE == 0) {
                            // bound pass: the k smallest upper bounds of this row's run
                            if (up < L[KL - 1]) {
                                float x = up;
#pragma unroll
                                for (int j = 0; j < KL; ++j) {
                                    const float a = fminf(L[j], x);
                                    x = fmaxf(L[j], x);
                                    L[j] = a;
                                }
                            }
                        } else if (lo <= T) {
                            // emit pass: the vector's lower bound is within T*
                            const int pos = atomicAdd(p.cnt + r, 1);
                            if (pos < p.cap) p.ent_id[r * p.cap + pos] = (int32_t)(cbase + i);
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty(b));
        }
        flush();
    }
    // ---- teardown ----
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TMEM_COLS) : "memory");
    }
    if (threadIdx.x == 0 && abort_flag) atomicExch(p.err, 1);
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ float tf32_rna(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// FP64 norm rounded up to FP32 (a bound used only inside margins)
__device__ __forceinline__ float norm_up(double sq) { return (float)sqrt(sq) * (1.f + 1.0f / 1048576.f); }

// Queries rounded to TF32 into the aligned operand buffer, with
// (||tf32(q)||, ||q - tf32(q)||); per-query state reset.
__global__ void dense_prep_kernel(const float *__restrict__ q, int64_t nq, int32_t d, float *__restrict__ qs,
                                  float2 *__restrict__ qnorm, int32_t *__restrict__ cnt, int32_t *__restrict__ ucnt,
                                  int32_t *__restrict__ err, unsigned long long *counters, int64_t n) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *err = 0;
        atomicAdd(counters + C_VALUES, (unsigned long long)nq * (unsigned long long)n * (unsigned long long)d);
        atomicAdd(counters + C_SCANNED, (unsigned long long)nq * (unsigned long long)n);
    }
    if (row >= nq) return;
    double st = 0.0, se = 0.0;
    for (int j = lane; j < d; j += 32) {
        const float v = q[row * d + j];
        const float t = tf32_rna(v);
        qs[row * d + j] = t;
        st += (double)t * t;
        se += ((double)v - t) * ((double)v - t);
    }
    st = warp_sum_f64(st);
    se = warp_sum_f64(se);
    if (lane == 0) {
        qnorm[row] = make_float2(norm_up(st), norm_up(se));
        cnt[row] = 0;
        ucnt[row] = 0;
    }
}

// Tensor-engine operand of the collection: rows rounded to TF32 and
// (||x||^2, ||x||, ||x - tf32(x)||, 0) from FP64 sums.
__global__ void dense_operand_kernel(const float *__restrict__ x, int64_t n, int32_t d, float *__restrict__ xtc,
                                     float4 *__restrict__ out) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    double sx = 0.0, se = 0.0;
    for (int j = lane; j < d; j += 32) {
        const float v = x[row * d + j];
        const float t = tf32_rna(v);
        xtc[row * d + j] = t;
        sx += (double)v * v;
        se += ((double)v - t) * ((double)v - t);
    }
    sx = warp_sum_f64(sx);
    se = warp_sum_f64(se);
    if (lane == 0) out[row] = make_float4((float)sx, norm_up(sx), norm_up(se), 0.f);
}

// T*[q] = k-th smallest value appended to ubuf[q]: a radix select over the
// order-preserving uint32 keys, 11 + 11 + 10 bits, one CTA per query. The
// runs partition the collection and each appended its k smallest upper
// bounds, so every vector among the k smallest upper bounds of the whole
// collection is there: this is the k-th smallest upper bound over all vectors
// (+inf when fewer than k were appended). If the buffer overflowed, the k-th
// of what it holds is larger, which only lengthens the candidate list.
__global__ void __launch_bounds__(256) dense_select_kernel(const float *__restrict__ ubuf, const int32_t *__restrict__ ucnt,
                                                           int32_t ucap, int32_t k, float *__restrict__ tstar) {
    __shared__ int hist[2048];
    __shared__ uint32_t s_prefix, s_want;
    const int64_t row = blockIdx.x;
    const float *u = ubuf + row * ucap;
    const int64_t L = min(ucnt[row], ucap);
    if (L < k) {  // fewer than k upper bounds: every vector is a candidate
        if (threadIdx.x == 0) tstar[row] = __int_as_float(0x7f800000);
        return;
    }
    uint32_t prefix = 0, mask = 0;
    if (threadIdx.x == 0) s_want = (uint32_t)k;
    const int shifts[3] = {21, 10, 0};
    const int widths[3] = {11, 11, 10};
    for (int pass = 0; pass < 3; ++pass) {
        const int sh = shifts[pass], nb = 1 << widths[pass];
        for (int i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < L; i += blockDim.x) {
            const uint32_t key = f2o(u[i]);
            if ((key & mask) == prefix) atomicAdd(&hist[(key >> sh) & (nb - 1)], 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t want = s_want, cum = 0;
            int bsel = nb - 1;
            for (int bi = 0; bi < nb; ++bi) {
                if (cum + (uint32_t)hist[bi] >= want) {
                    bsel = bi;
                    break;
                }
                cum += (uint32_t)hist[bi];
            }
            s_want = want - cum;
            s_prefix = prefix | ((uint32_t)bsel << sh);
        }
        __syncthreads();
        prefix = s_prefix;
        mask |= (uint32_t)(nb - 1) << sh;
        __syncthreads();
    }
    if (threadIdx.x == 0) tstar[row] = o2f(prefix);
}

// Block-wide ascending bitonic sort of buf[0..len), len a power of two.
__device__ void cta_bitonic(uint64_t *buf, int len) {
    for (int size = 2; size <= len; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < (len >> 1); i += blockDim.x) {
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

__device__ __forceinline__ int pow2_at_least(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Exact FP32 distance of query row qr to vector row xr: lane-strided
// dimensions and a fixed butterfly (the scan path's refine arithmetic).
template <int MET>
__device__ __forceinline__ float exact_dist(const float *qr, const float *xr, int d, int lane) {
    float acc = 0.f;
    for (int j = lane; j < d; j += 32) acc = term<MET>(qr[j], xr[j], acc);
    return rank_dist<MET>(warp_sum(acc));
}

struct FinishParams {
    int64_t nq, n;
    int32_t d, k, cap;
    const float *q;               // [nq][d]
    const float *x;               // [n][d]
    const int32_t *cnt;
    const int32_t *ent_id;
    const int32_t *err;
    uint64_t *out;                // [nq][k] keys
    unsigned long long *counters;
};

// One CTA per query: every emitted vector is a candidate (its lower bound is
// within T*); each gets its exact FP32 distance and the k best (distance, id)
// keys are kept.
template <int MET>
__global__ void __launch_bounds__(256) dense_finish_kernel(FinishParams f) {
    extern __shared__ __align__(16) uint64_t fbuf[];  // cap keys
    const int64_t row = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const float *qr = f.q + row * f.d;
    const int total = f.cnt[row];
    if (total > f.cap || *f.err) {
        // fallback: plain FP32 scan of all vectors, chunks merged into the best kpad
        const int kpad = pow2_at_least(f.k);
        const int chunk = f.cap - kpad;
        for (int i = tid; i < kpad; i += blockDim.x) fbuf[i] = kEmptyKey;
        for (int64_t off = 0; off < f.n; off += chunk) {
            for (int i = warp; i < chunk; i += nw) {
                const int64_t v = off + i;
                uint64_t key = kEmptyKey;
                if (v < f.n) key = make_key(exact_dist<MET>(qr, f.x + v * f.d, f.d, lane), (int32_t)v);
                if (lane == 0) fbuf[kpad + i] = key;
            }
            __syncthreads();
            cta_bitonic(fbuf, f.cap);
        }
        for (int i = tid; i < f.k; i += blockDim.x) f.out[row * f.k + i] = fbuf[i];
        if (tid == 0) atomicAdd(f.counters + C_DENSE_FALLBACK, 1ull);
        return;
    }
    const int32_t *eid = f.ent_id + row * f.cap;
    for (int c = warp; c < total; c += nw) {
        const int32_t id = eid[c];
        const float dist = exact_dist<MET>(qr, f.x + (int64_t)id * f.d, f.d, lane);
        if (lane == 0) fbuf[c] = make_key(dist, id);
    }
    const int len = pow2_at_least(total > f.k ? total : f.k);
    for (int i = total + tid; i < len; i += blockDim.x) fbuf[i] = kEmptyKey;
    __syncthreads();
    cta_bitonic(fbuf, len);
    for (int i = tid; i < f.k; i += blockDim.x) f.out[row * f.k + i] = fbuf[i];
    if (tid == 0) atomicAdd(f.counters + C_CANDIDATES, (unsigned long long)total);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) ==
                cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 2-D map over a row-major [rows][d] FP32 matrix, box of box_rows x 32
// elements, 128-byte swizzle, zero fill outside.
bool encode_rows(CUtensorMap *m, const float *base, int64_t rows, int32_t d, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)d * 4};
    cuuint32_t box[2] = {(cuuint32_t)TKF, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device, once per (kernel, device) and size (host-side cost only).
template <class K>
cudaError_t ensure_smem(K kernel, std::atomic<int> (&done)[64], int bytes) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::atomic<int> &have = done[dev & 63];
    if (have.load(std::memory_order_acquire) >= bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) {
        int cur = have.load();
        while (cur < bytes && !have.compare_exchange_weak(cur, bytes)) {
        }
    }
    return e;
}

template <int KL, int MET, int MODE>
cudaError_t launch_tc(const CUtensorMap &mq, const CUtensorMap &mx, const DenseParams &p, int grid, cudaStream_t st) {
    constexpr int EW = ew_for(KL);
    static std::atomic<int> done[64];
    cudaError_t e = ensure_smem(dense_tc_kernel<KL, MET, MODE, EW>, done, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    dense_tc_kernel<KL, MET, MODE, EW><<<grid, Epi<EW>::threads, SMEM_BYTES, st>>>(mq, mx, p);
    return counted(cudaGetLastError());
}

template <int MODE>
cudaError_t launch_tc_any(const CUtensorMap &mq, const CUtensorMap &mx, const DenseParams &p, int grid, int metric,
                          cudaStream_t st) {
    if (metric == MT_IP)
        return p.k <= 16 ? launch_tc<16, MT_IP, MODE>(mq, mx, p, grid, st) : launch_tc<64, MT_IP, MODE>(mq, mx, p, grid, st);
    return p.k <= 16 ? launch_tc<16, MT_L2, MODE>(mq, mx, p, grid, st) : launch_tc<64, MT_L2, MODE>(mq, mx, p, grid, st);
}

template <int MET>
cudaError_t launch_finish(const FinishParams &f, cudaStream_t st) {
    static std::atomic<int> done[64];
    const size_t smem = (size_t)f.cap * 8;
    cudaError_t e = ensure_smem(dense_finish_kernel<MET>, done, (int)smem);
    if (e != cudaSuccess) return e;
    dense_finish_kernel<MET><<<(unsigned)f.nq, 256, smem, st>>>(f);
    return counted(cudaGetLastError());
}

// Appended upper bounds per query: k per (CTA, column part) run; with the
// grid a multiple of the query tiles every CTA keeps one query tile, so
// grid * EW * k bounds the count (a smaller buffer would only loosen T*).
int32_t bound_cap(int sms, int32_t k) {
    const int64_t c = (int64_t)sms * ew_for(k <= 16 ? 16 : 64) * k;
    return (int32_t)std::min<int64_t>(std::max<int64_t>(c, 1024), 1 << 16);
}

// Persistent grid: a multiple of the query tiles (each CTA then serves one
// query tile), at most one CTA per SM.
int dense_grid(int64_t ntiles, int nqt, int sms) {
    int g = (int)std::min<int64_t>(ntiles, (int64_t)sms);
    if (nqt <= g) g -= g % nqt;
    return std::max(g, 1);
}

}  // namespace

bool dense_supported(const pdx_index *ix, int32_t k, const char **why) {
    const char *w = nullptr;
    if (ix->is_ivf) w = "the tensor-core engine serves exact indexes only";
    else if (!ix->xnary || !ix->xtc || !ix->xnorm) w = "the index keeps no tensor-engine operand (build with dense_rows=1)";
    else if (ix->metric != PDX_L2 && ix->metric != PDX_IP) w = "the tensor-core engine supports L2 and IP";
    else if (ix->d % 4 != 0) w = "the tensor-core engine needs d to be a multiple of 4 (16-byte rows for TMA)";
    else if (k > 64) w = "the tensor-core engine supports k <= 64";
    if (why) *why = w;
    return w == nullptr;
}

int dense_cap(int64_t n, int32_t k) {
    // candidates per query: the vectors whose lower bound is within the k-th
    // smallest upper bound; never more than the collection itself
    int64_t c = 4096;
    if (n < c) c = n;
    int p = 64;
    while (p < c) p <<= 1;
    while (p < 4 * k) p <<= 1;
    return p;
}

size_t dense_scratch_bytes(int64_t nq, int32_t d, int32_t k, int32_t cap, int64_t n, int sms) {
    auto rup = [](size_t b) { return (b + 255) & ~size_t(255); };
    return rup((size_t)nq * d * 4) + rup((size_t)nq * 8) + 3 * rup((size_t)nq * 4) +
           rup((size_t)nq * bound_cap(sms, k) * 4) +
           rup((size_t)nq * cap * 4) + rup((size_t)nq * k * 8) + rup(8);
}

pdx_status dense_run(const pdx_index *ix, const float *qd, int64_t nq, int32_t k, int metric, int out_mode,
                     unsigned char *scratch, size_t bytes, int cap, float *od, int64_t *oi, unsigned long long *counters,
                     int sms, void *ev_start, void *ev_stop, cudaStream_t st) {
    const int d = ix->d;
    const int32_t ucap = bound_cap(sms, k);
    auto rup = [](size_t b) { return (b + 255) & ~size_t(255); };
    size_t off = 0;
    auto take = [&](size_t b) {
        unsigned char *p = scratch + off;
        off += rup(b);
        return p;
    };
    float *qs = reinterpret_cast<float *>(take((size_t)nq * d * 4));
    float2 *qnorm = reinterpret_cast<float2 *>(take((size_t)nq * 8));
    float *tstar = reinterpret_cast<float *>(take((size_t)nq * 4));
    int32_t *cnt = reinterpret_cast<int32_t *>(take((size_t)nq * 4));
    int32_t *ucnt = reinterpret_cast<int32_t *>(take((size_t)nq * 4));
    float *ubuf = reinterpret_cast<float *>(take((size_t)nq * ucap * 4));
    int32_t *ent_id = reinterpret_cast<int32_t *>(take((size_t)nq * cap * 4));
    uint64_t *keys = reinterpret_cast<uint64_t *>(take((size_t)nq * k * 8));
    int32_t *err = reinterpret_cast<int32_t *>(take(8));
    if (off > bytes) {
        set_error("internal error: dense-search scratch layout exceeds its plan");
        return PDX_ERR_CUDA;
    }
    if (nq == 0) return PDX_OK;
    {
        const unsigned grid = (unsigned)((nq * 32 + 255) / 256);
        dense_prep_kernel<<<grid, 256, 0, st>>>(qd, nq, d, qs, qnorm, cnt, ucnt, err, counters, ix->n);
        cudaError_t e = counted(cudaGetLastError());
        if (e != cudaSuccess) return cuda_status_ext(e, "dense_prep_kernel");
    }
    CUtensorMap mq, mx;
    if (!encode_rows(&mq, qs, nq, d, TM) || !encode_rows(&mx, ix->xtc, ix->n, d, TN)) {
        set_error("cuTensorMapEncodeTiled failed (d=%d)", d);
        return PDX_ERR_CUDA;
    }
    DenseParams p;
    p.nq = nq;
    p.n = ix->n;
    p.d = d;
    p.k = k;
    p.nqt = (int32_t)((nq + TM - 1) / TM);
    p.ntiles = (int64_t)p.nqt * ((ix->n + TN - 1) / TN);
    p.qnorm = qnorm;
    p.xnorm = reinterpret_cast<const float4 *>(ix->xnorm);
    p.ubuf = ubuf;
    p.ucnt = ucnt;
    p.ucap = ucap;
    p.tstar = tstar;
    p.cnt = cnt;
    p.cap = cap;
    p.ent_id = ent_id;
    // margin coefficients (see dense_bounds): FP32 accumulation of D exact
    // products within (D+16) 2^-22 of sum |q~_j x~_j| (twice the sequential
    // bound, for an accumulation order we cannot see), a 2^-10 relative
    // cushion for the FP32 arithmetic of the margin itself
    const double u = std::ldexp(1.0, -22);
    const double cushion = 1.0 + std::ldexp(1.0, -10);
    p.k2 = (float)((metric == MT_L2 ? 2.0 : 1.0) * cushion);
    p.c_acc = (float)((d + 16) * u);
    p.c_xx = (float)(u);
    p.c_rel = (float)(4.0 * u);
    p.err = err;
    // test hook for the bounded waits (tests/test_gpu_dense.py): with
    // PDX_TEST_DENSE_STALL=1 no tile is loaded, every GEMM wait runs out after
    // its limit, the kernel releases TMEM and flags the error, and the finish
    // kernel answers every query by the plain FP32 scan
    const char *stall = std::getenv("PDX_TEST_DENSE_STALL");
    p.stall_test = (stall && stall[0] == '1') ? 1 : 0;
    const int grid = dense_grid(p.ntiles, p.nqt, sms);
    cudaError_t e;
    if (ev_start && (e = cudaEventRecord(static_cast<cudaEvent_t>(ev_start), st)) != cudaSuccess)
        return cuda_status_ext(e, "cudaEventRecord");
    // pass 1: per run, the k smallest upper bounds; then T* per query
    if ((e = launch_tc_any<0>(mq, mx, p, grid, metric, st)) != cudaSuccess)
        return cuda_status_ext(e, "dense_tc_kernel (bound pass)");
    dense_select_kernel<<<(unsigned)nq, 256, 0, st>>>(ubuf, ucnt, ucap, k, tstar);
    if ((e = counted(cudaGetLastError())) != cudaSuccess) return cuda_status_ext(e, "dense_select_kernel");
    // pass 2: emit the vectors whose lower bound is within T*
    if ((e = launch_tc_any<1>(mq, mx, p, grid, metric, st)) != cudaSuccess)
        return cuda_status_ext(e, "dense_tc_kernel (emit pass)");
    if (ev_stop && (e = cudaEventRecord(static_cast<cudaEvent_t>(ev_stop), st)) != cudaSuccess)
        return cuda_status_ext(e, "cudaEventRecord");
    FinishParams f;
    f.nq = nq;
    f.n = ix->n;
    f.d = d;
    f.k = k;
    f.cap = cap;
    f.q = qd;             // the rerank reads the exact FP32 queries and vectors
    f.x = ix->xnary;
    f.cnt = cnt;
    f.ent_id = ent_id;
    f.err = err;
    f.out = keys;
    f.counters = counters;
    e = metric == MT_IP ? launch_finish<MT_IP>(f, st) : launch_finish<MT_L2>(f, st);
    if (e != cudaSuccess) return cuda_status_ext(e, "dense_finish_kernel");
    e = launch_write_out(keys, nq, k, out_mode, qd, d, od, oi, st);
    if (e != cudaSuccess) return cuda_status_ext(e, "write_out_kernel");
    return PDX_OK;
}

cudaError_t launch_dense_operand(const float *x, int64_t n, int32_t d, float *xtc, float *out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    dense_operand_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(x, n, d, xtc,
                                                                           reinterpret_cast<float4 *>(out));
    return counted(cudaGetLastError());
}

}  // namespace pdx
