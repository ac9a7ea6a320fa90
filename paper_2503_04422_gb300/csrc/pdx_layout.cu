// Layout build (Sec. 3): N-ary rows -> PDX blocks, and block metadata.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "pdx_internal.cuh"

namespace pdx {

// One CTA transposes a 64-vector x 32-dimension tile through shared memory:
// rows are read 128 B at a time along dimensions (coalesced), and written
// 256 B at a time along vectors (coalesced), which is the PDX order
// data[(b*D + j)*64 + t]. Padding slots (id -1) are written as zeros.
__global__ void __launch_bounds__(256) to_pdx_kernel(const float *__restrict__ x, int32_t d,
                                                     const int32_t *__restrict__ ids,
                                                     float *__restrict__ data) {
    __shared__ float tile[kBlock][33];
    const int64_t b = blockIdx.x;
    const int j0 = blockIdx.y * 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < kBlock; r += 8) {
        int32_t id = ids[b * kBlock + r];
        int j = j0 + lane;
        float v = 0.f;
        if (id >= 0 && j < d) v = x[(int64_t)id * d + j];
        tile[r][lane] = v;
    }
    __syncthreads();
    for (int jj = warp; jj < 32; jj += 8) {
        int j = j0 + jj;
        if (j >= d) break;
        float *dst = data + ((b * d + j) * kBlock);
        dst[lane] = tile[lane][jj];
        dst[lane + 32] = tile[lane + 32][jj];
    }
}

cudaError_t launch_to_pdx(const float *x, int32_t d, const int32_t *ids, int64_t nblocks, float *data,
                          cudaStream_t st) {
    if (nblocks == 0) return cudaSuccess;
    dim3 grid((unsigned)nblocks, (unsigned)((d + 31) / 32));
    to_pdx_kernel<<<grid, 256, 0, st>>>(x, d, ids, data);
    return counted(cudaGetLastError());
}

// means[p][j] = average of dimension j over the valid vectors of part p
// (block metadata, Sec. 3; used by PDX-BOND's distance-to-means order, Sec. 5).
// One warp per (part, dimension): lanes cover the 64 slots of each block.
__global__ void part_means_kernel(const float *__restrict__ data, const int32_t *__restrict__ blk_cnt,
                                  const int32_t *__restrict__ part_blk, int32_t nparts, int32_t d,
                                  float *__restrict__ means) {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= (int64_t)nparts * d) return;
    const int p = (int)(gw / d), j = (int)(gw % d);
    float s = 0.f;
    int64_t cnt = 0;
    for (int b = part_blk[p]; b < part_blk[p + 1]; ++b) {
        const float *row = data + ((int64_t)b * d + j) * kBlock;
        int c = blk_cnt[b];
        if (lane < c) s += row[lane];
        if (lane + 32 < c) s += row[lane + 32];
        cnt += c;
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) means[(int64_t)p * d + j] = cnt ? s / (float)cnt : 0.f;
}

cudaError_t launch_part_means(const float *data, const int32_t *blk_cnt, const int32_t *part_blk,
                              int32_t nparts, int32_t d, float *means, cudaStream_t st) {
    int64_t warps = (int64_t)nparts * d;
    if (warps == 0) return cudaSuccess;
    part_means_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(data, blk_cnt, part_blk, nparts,
                                                                            d, means);
    return counted(cudaGetLastError());
}

// Population variance of every dimension over each part's vectors (the fused
// pruner's expected contributions), one warp per (part, dimension).
__global__ void part_vars_kernel(const float *__restrict__ data, const int32_t *__restrict__ blk_cnt,
                                 const int32_t *__restrict__ part_blk, int32_t nparts, int32_t d,
                                 const float *__restrict__ means, float *__restrict__ vars) {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= (int64_t)nparts * d) return;
    const int p = (int)(gw / d), j = (int)(gw % d);
    const float mu = means[(int64_t)p * d + j];
    float s = 0.f;
    int64_t cnt = 0;
    for (int b = part_blk[p]; b < part_blk[p + 1]; ++b) {
        const float *row = data + ((int64_t)b * d + j) * kBlock;
        const int c = blk_cnt[b];
        if (lane < c) {
            const float t = row[lane] - mu;
            s = fmaf(t, t, s);
        }
        if (lane + 32 < c) {
            const float t = row[lane + 32] - mu;
            s = fmaf(t, t, s);
        }
        cnt += c;
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) vars[(int64_t)p * d + j] = cnt ? s / (float)cnt : 0.f;
}

cudaError_t launch_part_vars(const float *data, const int32_t *blk_cnt, const int32_t *part_blk, int32_t nparts,
                             int32_t d, const float *means, float *vars, cudaStream_t st) {
    const int64_t warps = (int64_t)nparts * d;
    if (warps == 0) return cudaSuccess;
    part_vars_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(data, blk_cnt, part_blk, nparts, d, means,
                                                                           vars);
    return counted(cudaGetLastError());
}

// flag is cleared when some row's squared norm differs from 1 by more than tol.
__global__ void unit_norm_kernel(const float *__restrict__ x, int64_t n, int32_t d, float tol, int *flag) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    float s = 0.f;
    for (int j = lane; j < d; j += 32) {
        float v = x[row * d + j];
        s = fmaf(v, v, s);
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0 && fabsf(s - 1.f) > tol) atomicExch(flag, 0);
}

cudaError_t launch_unit_norm_check(const float *x, int64_t n, int32_t d, float tol, int *flag,
                                   cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    unit_norm_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(x, n, d, tol, flag);
    return counted(cudaGetLastError());
}

__global__ void fill_u32_kernel(uint32_t *p, uint32_t v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}
__global__ void fill_u64_kernel(uint64_t *p, uint64_t v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

cudaError_t launch_fill_u32(uint32_t *p, uint32_t v, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    fill_u32_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(p, v, n);
    return counted(cudaGetLastError());
}
cudaError_t launch_fill_u64(uint64_t *p, uint64_t v, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    fill_u64_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(p, v, n);
    return counted(cudaGetLastError());
}

__global__ void add_u64_kernel(unsigned long long *p, unsigned long long v) { atomicAdd(p, v); }

cudaError_t launch_add_u64(unsigned long long *p, unsigned long long v, cudaStream_t st) {
    add_u64_kernel<<<1, 1, 0, st>>>(p, v);
    return counted(cudaGetLastError());
}

// ---- low-precision storage ----
// colmax[j] = max_i |x_ij| as float bits (non-negative floats order like their bits)
__global__ void colmax_kernel(const float *__restrict__ x, int64_t n, int32_t d, unsigned *__restrict__ colmax) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    float m = 0.f;
    for (int64_t r = blockIdx.y; r < n; r += gridDim.y) m = fmaxf(m, fabsf(x[r * d + j]));
    atomicMax(colmax + j, __float_as_uint(m));
}

// scale[j] = colmax[j] / 448 (the largest E4M3 magnitude), 1 for an all-zero column
__global__ void fp8_scale_kernel(const unsigned *__restrict__ colmax, int32_t d, float *__restrict__ scale) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    float m = __uint_as_float(colmax[j]);
    scale[j] = m > 0.f ? m / 448.f : 1.f;
}

cudaError_t launch_fp8_scales(const float *x, int64_t n, int32_t d, unsigned *colmax, float *scale, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(colmax, 0, (size_t)d * 4, st);
    if (e != cudaSuccess) return e;
    dim3 g((unsigned)((d + 127) / 128), 256);
    colmax_kernel<<<g, 128, 0, st>>>(x, n, d, colmax);
    e = counted(cudaGetLastError());
    if (e != cudaSuccess) return e;
    fp8_scale_kernel<<<(unsigned)((d + 127) / 128), 128, 0, st>>>(colmax, d, scale);
    return counted(cudaGetLastError());
}

// Element-wise quantisation of the FP32 PDX blocks: BF16 round-to-nearest-even,
// or E4M3 (saturating, round-to-nearest-even) of x / scale[j].
__global__ void quantize_kernel(const float *__restrict__ data, int64_t total, int32_t d, int storage,
                                const float *__restrict__ scale, void *__restrict__ out) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const float x = data[t];
        if (storage == PDX_BF16) {
            static_cast<uint16_t *>(out)[t] = __bfloat16_as_ushort(__float2bfloat16_rn(x));
        } else {
            const int j = (int)((t / kBlock) % d);
            static_cast<uint8_t *>(out)[t] = (uint8_t)__nv_cvt_float_to_fp8(x / scale[j], __NV_SATFINITE, __NV_E4M3);
        }
    }
}

cudaError_t launch_quantize(const float *data, int64_t nblocks, int32_t d, int storage, const float *scale, void *out,
                            cudaStream_t st) {
    const int64_t total = nblocks * d * kBlock;
    if (total == 0) return cudaSuccess;
    int64_t blocks = (total + 255) / 256;
    quantize_kernel<<<(unsigned)(blocks < 8192 ? blocks : 8192), 256, 0, st>>>(data, total, d, storage, scale, out);
    return counted(cudaGetLastError());
}

}  // namespace pdx
