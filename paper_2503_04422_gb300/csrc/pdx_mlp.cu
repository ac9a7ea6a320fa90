// Order-proposal network for PDX-BOND (no counterpart in the paper): a
// 2-layer MLP u = [q; c] (2D) -> relu (H) -> D scores, trained on the GPU with
// these kernels (FP32 master weights, Adam), run for inference with BF16
// copies of the weights (FP32 accumulate). Its scores order the dimensions a
// search visits; the prune test stays the true partial distance, so results
// are exact whatever the network proposes.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "pdx_internal.cuh"


namespace pdx {

// ---------------------------------------------------------------------------
// C[M][N] = alpha * op(A) op(B) + beta * C, row-major. op(A) is M x K (A
// stored M x K, or K x M when TA), op(B) is K x N (B stored K x N, or N x K
// when TB); B may hold BF16 bits (inference weights). 64 x 64 tiles, 32-deep
// k-chunks in shared memory, 4 x 4 outputs per thread, FP32 accumulate.
template <bool TA, bool TB, typename BT>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float *__restrict__ A, int lda,
                                                   const BT *__restrict__ B, int ldb, float *__restrict__ C, int ldc,
                                                   float alpha, float beta) {
    __shared__ __align__(16) float As[32][68];
    __shared__ __align__(16) float Bs[32][68];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 32) {
        for (int e = tid; e < 64 * 32; e += 256) {
            int r = e >> 5, kk = e & 31;    // (row of the tile, k)
            int mm = m0 + r, k = k0 + kk;
            float a = 0.f;
            if (mm < M && k < K) a = TA ? A[(size_t)k * lda + mm] : A[(size_t)mm * lda + k];
            As[kk][r] = a;
            int nn = n0 + r;
            float b = 0.f;
            if (nn < N && k < K) {
                BT raw = TB ? B[(size_t)nn * ldb + k] : B[(size_t)k * ldb + nn];
                if constexpr (sizeof(BT) == 2)
                    b = __uint_as_float((uint32_t)raw << 16);
                else
                    b = raw;
            }
            Bs[kk][r] = b;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 32; ++kk) {
            float4 a = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
            float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
            float aa[4] = {a.x, a.y, a.z, a.w}, bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(aa[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int mm = m0 + ty * 4 + i;
        if (mm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int nn = n0 + tx * 4 + j;
            if (nn >= N) continue;
            float *c = C + (size_t)mm * ldc + nn;
            *c = alpha * acc[i][j] + (beta != 0.f ? beta * *c : 0.f);
        }
    }
}

template <bool TA, bool TB, typename BT>
static cudaError_t gemm(int M, int N, int K, const float *A, int lda, const BT *B, int ldb, float *C, int ldc,
                        float alpha, float beta, cudaStream_t st) {
    if (M == 0 || N == 0) return cudaSuccess;
    if ((M + 63) / 64 > 65535) return cudaErrorInvalidValue;  // grid.y limit
    dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64));
    gemm_kernel<TA, TB, BT><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta);
    return counted(cudaGetLastError());
}

// Z[r][j] += b[j]; with H: H = act(Z) and Z keeps the pre-activation (training);
// without H: Z = act(Z + b) in place (inference)
__global__ void bias_act_kernel(float *Z, float *H, const float *__restrict__ b, int64_t rows, int cols, int relu) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * cols) return;
    float z = Z[t] + b[t % cols];
    float a = relu ? fmaxf(z, 0.f) : z;
    if (H) {
        Z[t] = z;
        H[t] = a;
    } else {
        Z[t] = a;
    }
}

// dY = 2 (Y - T) / (B*D); loss partial sums of (Y - T)^2
__global__ void mse_grad_kernel(const float *__restrict__ Y, const float *__restrict__ T, int64_t total, float scale,
                                float *__restrict__ dY, double *__restrict__ loss) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float e = 0.f;
    if (t < total) {
        float r = Y[t] - T[t];
        dY[t] = 2.f * r * scale;
        e = r * r;
    }
    for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0 && e != 0.f) atomicAdd(loss, (double)e);
}

// dZ = dH * (Z > 0)
__global__ void relu_back_kernel(float *__restrict__ dH, const float *__restrict__ Z, int64_t total) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < total && !(Z[t] > 0.f)) dH[t] = 0.f;
}

// out[j] = sum_r X[r][j]
__global__ void colsum_f_kernel(const float *__restrict__ X, int64_t rows, int cols, float *__restrict__ out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float s = 0.f;
    for (int64_t r = 0; r < rows; ++r) s += X[r * cols + j];
    out[j] = s;
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, size_t n, float lr, float b1, float b2, float c1, float c2,
                            float eps) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void to_bf16_kernel(const float *__restrict__ x, uint16_t *__restrict__ y, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __bfloat16_as_ushort(__float2bfloat16_rn(x[i]));
}

// rows of U and T gathered by a permutation (one CTA per row)
__global__ void gather_rows_kernel(const float *__restrict__ src, const int32_t *__restrict__ idx, int cols,
                                   float *__restrict__ dst) {
    const int64_t r = blockIdx.x;
    const float *s = src + (int64_t)idx[r] * cols;
    for (int j = threadIdx.x; j < cols; j += blockDim.x) dst[r * cols + j] = s[j];
}

static inline unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

struct MlpWork {
    float *Z, *H, *Y, *dY, *dH;
    double *loss;
};

// Forward on B rows of U ([B][2D]) into Y ([B][D]); keeps Z, H for backward.
static cudaError_t mlp_forward_impl(const pdx_mlp *net, const float *U, int64_t B, bool bf16, float *Z, float *H,
                                    float *Y, cudaStream_t st) {
    const int D = net->d, Hn = net->hidden, IN = 2 * net->d;
    cudaError_t e;
    if (bf16)
        e = gemm<false, true, uint16_t>((int)B, Hn, IN, U, IN, net->w1h, IN, Z, Hn, 1.f, 0.f, st);
    else
        e = gemm<false, true, float>((int)B, Hn, IN, U, IN, net->w1(), IN, Z, Hn, 1.f, 0.f, st);
    if (e != cudaSuccess) return e;
    bias_act_kernel<<<blocks_for(B * Hn), 256, 0, st>>>(Z, (H == Z) ? nullptr : H, net->b1(), B, Hn, 1);
    if ((e = counted(cudaGetLastError())) != cudaSuccess) return e;
    if (bf16)
        e = gemm<false, true, uint16_t>((int)B, D, Hn, H, Hn, net->w2h, Hn, Y, D, 1.f, 0.f, st);
    else
        e = gemm<false, true, float>((int)B, D, Hn, H, Hn, net->w2(), Hn, Y, D, 1.f, 0.f, st);
    if (e != cudaSuccess) return e;
    bias_act_kernel<<<blocks_for(B * D), 256, 0, st>>>(Y, nullptr, net->b2(), B, D, 0);
    return counted(cudaGetLastError());
}

// Backward of the MSE loss into net->g; loss sum (not normalised) into *loss.
static cudaError_t mlp_backward_impl(pdx_mlp *net, const float *U, const float *T, int64_t B, const MlpWork &w,
                                     cudaStream_t st) {
    const int D = net->d, Hn = net->hidden, IN = 2 * net->d;
    cudaError_t e = mlp_forward_impl(net, U, B, false, w.Z, w.H, w.Y, st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.loss, 0, 8, st)) != cudaSuccess) return e;
    mse_grad_kernel<<<blocks_for(B * D), 256, 0, st>>>(w.Y, T, B * D, 1.f / (float)(B * D), w.dY, w.loss);
    if ((e = counted(cudaGetLastError())) != cudaSuccess) return e;
    float *gW1 = net->g, *gb1 = gW1 + (size_t)Hn * IN, *gW2 = gb1 + Hn, *gb2 = gW2 + (size_t)D * Hn;
    // dW2 = dY^T H  [D][H]
    if ((e = gemm<true, false, float>(D, Hn, (int)B, w.dY, D, w.H, Hn, gW2, Hn, 1.f, 0.f, st)) != cudaSuccess) return e;
    colsum_f_kernel<<<blocks_for(D), 256, 0, st>>>(w.dY, B, D, gb2);
    if ((e = counted(cudaGetLastError())) != cudaSuccess) return e;
    // dH = dY W2  [B][H], then dZ = dH * (Z > 0)
    if ((e = gemm<false, false, float>((int)B, Hn, D, w.dY, D, net->w2(), Hn, w.dH, Hn, 1.f, 0.f, st)) != cudaSuccess)
        return e;
    relu_back_kernel<<<blocks_for(B * Hn), 256, 0, st>>>(w.dH, w.Z, B * Hn);
    if ((e = counted(cudaGetLastError())) != cudaSuccess) return e;
    // dW1 = dZ^T U  [H][2D]; db1 = colsum(dZ)
    if ((e = gemm<true, false, float>(Hn, IN, (int)B, w.dH, Hn, U, IN, gW1, IN, 1.f, 0.f, st)) != cudaSuccess) return e;
    colsum_f_kernel<<<blocks_for(Hn), 256, 0, st>>>(w.dH, B, Hn, gb1);
    return counted(cudaGetLastError());
}

static cudaError_t refresh_bf16(pdx_mlp *net, cudaStream_t st) {
    if (!net->bf16_stale) return cudaSuccess;
    size_t n1 = (size_t)net->hidden * 2 * net->d, n2 = (size_t)net->d * net->hidden;
    to_bf16_kernel<<<blocks_for((int64_t)n1), 256, 0, st>>>(net->w1(), net->w1h, n1);
    cudaError_t e = counted(cudaGetLastError());
    if (e != cudaSuccess) return e;
    to_bf16_kernel<<<blocks_for((int64_t)n2), 256, 0, st>>>(net->w2(), net->w2h, n2);
    e = counted(cudaGetLastError());
    if (e == cudaSuccess) net->bf16_stale = false;
    return e;
}

// Inference for a search: Y [B][D] scores from U [B][2D] with the BF16 weights.
cudaError_t mlp_scores(pdx_mlp *net, const float *U, int64_t B, float *Z, float *Y, cudaStream_t st) {
    cudaError_t e = refresh_bf16(net, st);
    if (e != cudaSuccess) return e;
    return mlp_forward_impl(net, U, B, true, Z, Z, Y, st);
}



// ---------------------------------------------------------------------------
// The learned visit order in one launch ahead of the scan: one CTA per query
// builds u = [q; c] (c: the nearest centroid, from its key), runs both layers
// with the BF16 weights and FP32 accumulation (a warp per output: lanes take
// pairs of BF16 weights, then a warp sum), adds the biases and the ReLU, forms
// the score (q_j - mu_j)^2 + s_q y_j (mu: collection means, s_q: the query's
// mean heuristic term), and sorts the dimensions by decreasing score (ties to
// the lower dimension) into the query's row of the order array.
__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

__global__ void __launch_bounds__(256) mlp_order_kernel(const float *__restrict__ q, int64_t nq, int d, int H,
                                                        const float *__restrict__ cent,
                                                        const uint64_t *__restrict__ nearest,
                                                        const uint16_t *__restrict__ w1h, const float *__restrict__ b1,
                                                        const uint16_t *__restrict__ w2h, const float *__restrict__ b2,
                                                        const float *__restrict__ mu, uint16_t *__restrict__ order) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int64_t r = blockIdx.x;
    if (r >= nq) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int npad = [&] { int p = 1; while (p < d) p <<= 1; return p; }();
    uint64_t *keys = reinterpret_cast<uint64_t *>(sm);       // [npad]
    float *u = reinterpret_cast<float *>(keys + npad);       // [2d]
    float *h = u + 2 * d;                                    // [H]
    __shared__ float red[32];
    const int c = (int)(uint32_t)(nearest[r] & 0xffffffffu);
    float part = 0.f;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const float qj = q[r * d + j];
        u[j] = qj;
        u[d + j] = cent[(int64_t)c * d + j];
        const float t = qj - mu[j];
        part = fmaf(t, t, part);
    }
    for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    float sq = 0.f;
    for (int i = 0; i < nw; ++i) sq += red[i];
    sq /= (float)d;
    // layer 1: h = relu(W1 u + b1), W1 [H][2d] in BF16 (2d even: pairs of weights)
    for (int o = warp; o < H; o += nw) {
        const uint32_t *wr = reinterpret_cast<const uint32_t *>(w1h + (int64_t)o * 2 * d);
        float acc = 0.f;
        for (int i = lane; i < d; i += 32) {
            const uint32_t w = __ldg(wr + i);
            acc = fmaf(bf16_lo(w), u[2 * i], acc);
            acc = fmaf(bf16_hi(w), u[2 * i + 1], acc);
        }
        for (int s = 16; s; s >>= 1) acc += __shfl_xor_sync(kFull, acc, s);
        if (lane == 0) h[o] = fmaxf(acc + b1[o], 0.f);
    }
    __syncthreads();
    // layer 2 and the score: y = W2 h + b2, W2 [d][H] in BF16 (H even)
    for (int j = warp; j < npad; j += nw) {
        uint64_t key = kEmptyKey;
        if (j < d) {
            const uint32_t *wr = reinterpret_cast<const uint32_t *>(w2h + (int64_t)j * H);
            float acc = 0.f;
            for (int i = lane; i < H / 2; i += 32) {
                const uint32_t w = __ldg(wr + i);
                acc = fmaf(bf16_lo(w), h[2 * i], acc);
                acc = fmaf(bf16_hi(w), h[2 * i + 1], acc);
            }
            for (int s = 16; s; s >>= 1) acc += __shfl_xor_sync(kFull, acc, s);
            const float t = u[j] - mu[j];
            const float sc = fmaf(t, t, sq * (acc + b2[j]));
            key = ((uint64_t)f2o(-sc) << 32) | (uint32_t)j;
        }
        if (lane == 0) keys[j] = key;
    }
    __syncthreads();
    for (int size = 2; size <= npad; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < (npad >> 1); i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
                const bool asc = (lo & size) == 0;
                const uint64_t a = keys[lo], b = keys[hi];
                if ((a > b) == asc) {
                    keys[lo] = b;
                    keys[hi] = a;
                }
            }
            __syncthreads();
        }
    }
    for (int j = threadIdx.x; j < d; j += blockDim.x) order[r * d + j] = (uint16_t)(keys[j] & 0xffffu);
}

cudaError_t mlp_order(pdx_mlp *net, const float *q, int64_t nq, const float *cent, const uint64_t *nearest,
                      const float *mu, uint16_t *order, cudaStream_t st) {
    if (nq == 0) return cudaSuccess;
    cudaError_t e = refresh_bf16(net, st);
    if (e != cudaSuccess) return e;
    const int d = net->d, H = net->hidden;
    int npad = 1;
    while (npad < d) npad <<= 1;
    const size_t smem = (size_t)npad * 8 + (size_t)(2 * d + H) * 4;
    if ((e = raise_smem_limit(mlp_order_kernel, smem)) != cudaSuccess) return e;
    mlp_order_kernel<<<(unsigned)nq, 256, smem, st>>>(q, nq, d, H, cent, nearest, net->w1h, net->b1(), net->w2h,
                                                       net->b2(), mu, order);
    return counted(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// u[r] = [q_r; c_(a_r)] with a_r the centroid id in keys[r] (nearest centroid)
__global__ void mlp_inputs_kernel(const float *__restrict__ q, int64_t nq, int d, const float *__restrict__ cent,
                                  const uint64_t *__restrict__ nearest, float *__restrict__ u) {
    const int64_t r = blockIdx.x;
    if (r >= nq) return;
    const int c = (int)(uint32_t)(nearest[r] & 0xffffffffu);
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        u[r * 2 * d + j] = q[r * d + j];
        u[r * 2 * d + d + j] = cent[(int64_t)c * d + j];
    }
}

cudaError_t launch_mlp_inputs(const float *q, int64_t nq, int d, const float *cent, const uint64_t *nearest, float *u,
                              cudaStream_t st) {
    if (nq == 0) return cudaSuccess;
    mlp_inputs_kernel<<<(unsigned)nq, 256, 0, st>>>(q, nq, d, cent, nearest, u);
    return counted(cudaGetLastError());
}

// Trace targets: t[r][j] = mean over the m vectors ids[r][*] of (q_rj - x_j)^2
// minus the heuristic term (q_rj - mu_j)^2 (mu = collection means), in units of
// s_q = mean_j (q_rj - mu_j)^2. The ids
// are vectors the plain search had to prune for query r: a sample of the
// collection plus the ones it ranked just behind the top-k, which survive
// longest. Visiting first the dimensions where they differ most from q prunes
// them soonest; the network learns the part of that the heuristic misses.
__global__ void targets_kernel(const float *__restrict__ q, int64_t nq, int d, const int64_t *__restrict__ ids, int m,
                               const float *__restrict__ data, const float *__restrict__ xnary,
                               const int32_t *__restrict__ slot_of, const float *__restrict__ mu,
                               float *__restrict__ t) {
    const int64_t r = blockIdx.x;
    __shared__ float red[256];
    float part = 0.f;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        float t0 = q[r * d + j] - mu[j];
        part = fmaf(t0, t0, part);
    }
    red[threadIdx.x] = part;
    __syncthreads();
    for (int o = blockDim.x >> 1; o; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const float sq = red[0] / (float)d;  // s_q = mean_j (q_j - mu_j)^2: the unit of the targets
    const float inv = sq > 0.f ? 1.f / sq : 0.f;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const float qj = q[r * d + j];
        float s = 0.f;
        int cnt = 0;
        for (int i = 0; i < m; ++i) {
            const int64_t id = ids[r * m + i];
            if (id < 0) continue;
            float x;
            if (xnary) {
                x = xnary[id * d + j];
            } else {
                const int slot = slot_of[id];
                x = data[((int64_t)(slot / kBlock) * d + j) * kBlock + (slot % kBlock)];
            }
            float df = qj - x;
            s = fmaf(df, df, s);
            ++cnt;
        }
        const float h = (qj - mu[j]) * (qj - mu[j]);
        t[r * d + j] = ((cnt ? s / (float)cnt : h) - h) * inv;
    }
}

}  // namespace pdx

using namespace pdx;

static pdx_status mlp_err(cudaError_t e, const char *what) { return cuda_status_ext(e, what); }

extern "C" size_t pdx_mlp_param_count(const pdx_mlp *net) { return net ? net->count : 0; }

extern "C" void pdx_mlp_free(pdx_mlp *net) {
    if (!net) return;
    void *ptrs[] = {net->p, net->g, net->m, net->v, net->w1h, net->w2h};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    delete net;
}

extern "C" pdx_status pdx_mlp_create(int32_t d, int32_t hidden, uint64_t seed, pdx_mlp **out) {
    if (out) *out = nullptr;
    if (!out || d < 1 || d > kMaxD || hidden < 1 || hidden > 4096) {
        set_error("pdx_mlp_create: d=%d hidden=%d out of range", d, hidden);
        return PDX_ERR_ARG;
    }
    pdx_mlp *net = new (std::nothrow) pdx_mlp();
    if (!net) return PDX_ERR_OOM;
    net->d = d;
    net->hidden = hidden;
    const size_t n1 = (size_t)hidden * 2 * d, n2 = (size_t)d * hidden;
    net->count = n1 + hidden + n2 + d;
    cudaError_t e = cudaMalloc(&net->p, net->count * 4);
    if (e == cudaSuccess) e = cudaMalloc(&net->g, net->count * 4);
    if (e == cudaSuccess) e = cudaMalloc(&net->m, net->count * 4);
    if (e == cudaSuccess) e = cudaMalloc(&net->v, net->count * 4);
    if (e == cudaSuccess) e = cudaMalloc(&net->w1h, n1 * 2);
    if (e == cudaSuccess) e = cudaMalloc(&net->w2h, n2 * 2);
    if (e != cudaSuccess) {
        pdx_mlp_free(net);
        return mlp_err(e, "pdx_mlp_create");
    }
    // Glorot-uniform weights from splitmix64, zero biases
    std::vector<float> h(net->count, 0.f);
    uint64_t s = seed;
    auto uni = [&]() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    const double a1 = std::sqrt(6.0 / (2.0 * d + hidden)), a2 = std::sqrt(6.0 / ((double)hidden + d));
    for (size_t i = 0; i < n1; ++i) h[i] = (float)((2 * uni() - 1) * a1);
    for (size_t i = 0; i < n2; ++i) h[n1 + hidden + i] = (float)((2 * uni() - 1) * a2);
    e = cudaMemcpy(net->p, h.data(), net->count * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(net->m, 0, net->count * 4);
    if (e == cudaSuccess) e = cudaMemset(net->v, 0, net->count * 4);
    if (e != cudaSuccess) {
        pdx_mlp_free(net);
        return mlp_err(e, "pdx_mlp_create");
    }
    *out = net;
    return PDX_OK;
}

extern "C" pdx_status pdx_mlp_set_params(pdx_mlp *net, const float *params, size_t count) {
    if (!net || !params || count != net->count) {
        set_error("pdx_mlp_set_params: NULL argument or count %zu != %zu", count, net ? net->count : 0);
        return PDX_ERR_ARG;
    }
    cudaError_t e = cudaMemcpy(net->p, params, count * 4, cudaMemcpyDefault);
    if (e != cudaSuccess) return mlp_err(e, "pdx_mlp_set_params");
    net->bf16_stale = true;
    return PDX_OK;
}

extern "C" pdx_status pdx_mlp_get_params(const pdx_mlp *net, float *params, size_t count) {
    if (!net || !params || count != net->count) {
        set_error("pdx_mlp_get_params: NULL argument or count %zu != %zu", count, net ? net->count : 0);
        return PDX_ERR_ARG;
    }
    cudaError_t e = cudaMemcpy(params, net->p, count * 4, cudaMemcpyDefault);
    return e == cudaSuccess ? PDX_OK : mlp_err(e, "pdx_mlp_get_params");
}

namespace {
struct Buf {
    void *p = nullptr;
    ~Buf() {
        if (p) cudaFree(p);
    }
};
}  // namespace

extern "C" pdx_status pdx_mlp_forward(pdx_mlp *net, const float *u, int64_t B, int32_t use_bf16, float *y,
                                      void *stream) {
    if (!net || (B > 0 && (!u || !y)) || B < 0 || B > (1 << 24)) {
        set_error("pdx_mlp_forward: bad argument");
        return PDX_ERR_ARG;
    }
    if (B == 0) return PDX_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Buf z;
    cudaError_t e = cudaMalloc(&z.p, (size_t)B * net->hidden * 4);
    if (e == cudaSuccess && use_bf16) e = refresh_bf16(net, st);
    if (e == cudaSuccess)
        e = mlp_forward_impl(net, u, B, use_bf16 != 0, (float *)z.p, (float *)z.p, y, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? PDX_OK : mlp_err(e, "pdx_mlp_forward");
}

extern "C" pdx_status pdx_mlp_backward(pdx_mlp *net, const float *u, const float *t, int64_t B, float *grads,
                                       float *loss_out, void *stream) {
    if (!net || !u || !t || !grads || B < 1 || B > (1 << 24)) {
        set_error("pdx_mlp_backward: bad argument");
        return PDX_ERR_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int D = net->d, Hn = net->hidden;
    Buf wb;
    size_t need = ((size_t)B * Hn * 3 + (size_t)B * D * 2) * 4 + 64;
    cudaError_t e = cudaMalloc(&wb.p, need);
    if (e != cudaSuccess) return mlp_err(e, "pdx_mlp_backward");
    float *base = (float *)wb.p;
    MlpWork w{base, base + (size_t)B * Hn, base + (size_t)B * Hn * 2, base + (size_t)B * Hn * 2 + (size_t)B * D,
              base + (size_t)B * Hn * 2 + (size_t)B * D * 2, nullptr};
    w.loss = reinterpret_cast<double *>(((uintptr_t)(w.dH + (size_t)B * Hn) + 15) & ~(uintptr_t)15);
    e = mlp_backward_impl(net, u, t, B, w, st);
    double ls = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(grads, net->g, net->count * 4, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ls, w.loss, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return mlp_err(e, "pdx_mlp_backward");
    if (loss_out) *loss_out = (float)(ls / ((double)B * D));
    return PDX_OK;
}

extern "C" pdx_status pdx_mlp_train(pdx_mlp *net, const float *u, const float *t, int64_t n, int32_t epochs,
                                    int32_t batch, float lr, uint64_t seed, float *loss_out, void *stream) {
    if (!net || !u || !t || n < 1 || epochs < 1 || batch < 1 || batch > 65536 || !(lr > 0.f)) {
        set_error("pdx_mlp_train: bad argument");
        return PDX_ERR_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int D = net->d, Hn = net->hidden, IN = 2 * D;
    const int64_t B = std::min<int64_t>(batch, n);
    Buf wb, ub, ib;
    size_t need = ((size_t)B * Hn * 3 + (size_t)B * D * 3) * 4 + 64;
    cudaError_t e = cudaMalloc(&wb.p, need);
    if (e == cudaSuccess) e = cudaMalloc(&ub.p, (size_t)B * IN * 4);
    if (e == cudaSuccess) e = cudaMalloc(&ib.p, (size_t)n * 4);
    if (e != cudaSuccess) return mlp_err(e, "pdx_mlp_train");
    float *base = (float *)wb.p;
    MlpWork w{base, base + (size_t)B * Hn, base + (size_t)B * Hn * 2, base + (size_t)B * Hn * 2 + (size_t)B * D,
              base + (size_t)B * Hn * 2 + (size_t)B * D * 2, nullptr};
    float *Tb = w.dH + (size_t)B * Hn;
    w.loss = reinterpret_cast<double *>(((uintptr_t)(Tb + (size_t)B * D) + 15) & ~(uintptr_t)15);
    std::vector<int32_t> perm((size_t)n);
    uint64_t s = seed;
    auto next = [&]() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    double last = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int64_t i = 0; i < n; ++i) perm[(size_t)i] = (int32_t)i;
        for (int64_t i = n - 1; i > 0; --i) std::swap(perm[(size_t)i], perm[(size_t)(next() % (uint64_t)(i + 1))]);
        if ((e = cudaMemcpyAsync(ib.p, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
        double ep_loss = 0.0;
        int64_t steps = 0;
        for (int64_t b0 = 0; b0 + B <= n; b0 += B) {
            const int32_t *idx = (const int32_t *)ib.p + b0;
            gather_rows_kernel<<<(unsigned)B, 256, 0, st>>>(u, idx, IN, (float *)ub.p);
            if ((e = counted(cudaGetLastError())) != cudaSuccess) break;
            gather_rows_kernel<<<(unsigned)B, 256, 0, st>>>(t, idx, D, Tb);
            if ((e = counted(cudaGetLastError())) != cudaSuccess) break;
            if ((e = mlp_backward_impl(net, (const float *)ub.p, Tb, B, w, st)) != cudaSuccess) break;
            net->adam_t += 1;
            const float c1 = 1.f - std::pow(0.9f, (float)net->adam_t), c2 = 1.f - std::pow(0.999f, (float)net->adam_t);
            adam_kernel<<<blocks_for((int64_t)net->count), 256, 0, st>>>(net->p, net->g, net->m, net->v, net->count, lr,
                                                                        0.9f, 0.999f, c1, c2, 1e-8f);
            if ((e = counted(cudaGetLastError())) != cudaSuccess) break;
            if (b0 + 2 * B > n) {  // last batch of the epoch: read its loss
                double ls = 0.0;
                if ((e = cudaMemcpyAsync(&ls, w.loss, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
                if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
                ep_loss = ls / ((double)B * D);
            }
            ++steps;
        }
        if (e != cudaSuccess) break;
        last = ep_loss;
    }
    net->bf16_stale = true;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return mlp_err(e, "pdx_mlp_train");
    if (loss_out) *loss_out = (float)last;
    return PDX_OK;
}

extern "C" pdx_status pdx_mlp_inputs(const float *q, int64_t nq, int32_t d, const float *centroids, int32_t nc,
                                      float *u, void *stream) {
    if (!q || !centroids || !u || nq < 0 || d < 1 || nc < 1) {
        set_error("pdx_mlp_inputs: bad argument");
        return PDX_ERR_ARG;
    }
    if (nq == 0) return PDX_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t Lc = ((int64_t)nc + kBlock - 1) / kBlock * kBlock;
    Buf kb, nb;
    cudaError_t e = cudaMalloc(&kb.p, (size_t)nq * Lc * 8);
    if (e == cudaSuccess) e = cudaMalloc(&nb.p, (size_t)nq * 8);
    if (e == cudaSuccess) e = launch_fill_u64((uint64_t *)kb.p, kEmptyKey, nq * Lc, st);
    if (e == cudaSuccess) e = launch_dense_keys_rows(q, nq, centroids, nc, d, Lc, (uint64_t *)kb.p, st);
    if (e == cudaSuccess) e = launch_select_k((uint64_t *)kb.p, nq, Lc, 1, (uint64_t *)nb.p, st);
    if (e == cudaSuccess) e = launch_mlp_inputs(q, nq, d, centroids, (uint64_t *)nb.p, u, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? PDX_OK : mlp_err(e, "pdx_mlp_inputs");
}

extern "C" pdx_status pdx_order_targets(const pdx_index *ix, const float *q, int64_t nq, const int64_t *ids, int32_t m,
                                        float *targets, void *stream) {
    if (!ix || !q || !ids || !targets || nq < 0 || m < 1) {
        set_error("pdx_order_targets: bad argument");
        return PDX_ERR_ARG;
    }
    if (nq == 0) return PDX_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    targets_kernel<<<(unsigned)nq, 256, 0, st>>>(q, nq, ix->d, ids, m, ix->data, ix->xnary, ix->slot_of, ix->cmean,
                                                 targets);
    cudaError_t e = counted(cudaGetLastError());
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? PDX_OK : mlp_err(e, "pdx_order_targets");
}
