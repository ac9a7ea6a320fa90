// IVF index on the GPU (Sec. 2.1, Fig. 2): transforms (ADSampling rotation,
// BSA PCA projection, Sec. 2.3), Lloyd k-means, nearest-centroid assignment,
// bucket probing, and the per-block metadata BSA needs.
#include "pdx_internal.cuh"

namespace pdx {

// ---------------------------------------------------------------------------
// y[r][i] = sum_j M[i][j] * (x[r][j] - shift[j])  (FP32, 128 x 64 output
// tiles, 16-dimension k-chunks staged in shared memory with the next chunk
// loaded into registers meanwhile, 8 x 4 outputs per thread; every output is
// summed in dimension order)
__global__ void __launch_bounds__(256) transform_kernel(const float *__restrict__ x, int64_t rows, int32_t d,
                                                        const float *__restrict__ M, const float *__restrict__ shift,
                                                        float *__restrict__ y) {
    constexpr int TR = 128, TI = 64, KC = 16;
    __shared__ __align__(16) float Xs[KC][TR + 4];
    __shared__ __align__(16) float Ms[KC][TI + 4];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;  // rows ty*8..+7, outputs tx*4..+3
    const int64_t r0 = (int64_t)blockIdx.x * TR;
    const int i0 = blockIdx.y * TI;
    float acc[8][4];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
    float xpf[8], mpf[4];
    auto load = [&](int j0) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = tid + 256 * u;
            const int rr = e >> 4, jj = e & 15;
            const int64_t r = r0 + rr;
            const int j = j0 + jj;
            xpf[u] = (r < rows && j < d) ? x[r * d + j] - (shift ? shift[j] : 0.f) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = tid + 256 * u;
            const int ii = e >> 4, jj = e & 15;
            const int i = i0 + ii, j = j0 + jj;
            mpf[u] = (i < d && j < d) ? M[(int64_t)i * d + j] : 0.f;
        }
    };
    load(0);
    for (int j0 = 0; j0 < d; j0 += KC) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = tid + 256 * u;
            Xs[e & 15][e >> 4] = xpf[u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = tid + 256 * u;
            Ms[e & 15][e >> 4] = mpf[u];
        }
        __syncthreads();
        if (j0 + KC < d) load(j0 + KC);
        const int jn = min(KC, d - j0);
        for (int jj = 0; jj < jn; ++jj) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&Xs[jj][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&Xs[jj][ty * 8 + 4]);
            const float4 bv = *reinterpret_cast<const float4 *>(&Ms[jj][tx * 4]);
            const float aa[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(aa[u], bb[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int64_t r = r0 + ty * 8 + u;
        if (r >= rows) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = i0 + tx * 4 + v;
            if (i < d) y[r * d + i] = acc[u][v];
        }
    }
}

cudaError_t launch_transform(const float *x, int64_t rows, int32_t d, const float *M, const float *shift, float *y,
                             cudaStream_t st) {
    if (rows == 0) return cudaSuccess;
    dim3 grid((unsigned)((rows + 127) / 128), (unsigned)((d + 63) / 64));
    transform_kernel<<<grid, 256, 0, st>>>(x, rows, d, M, shift, y);
    return counted(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Nearest centroid of every row (L2, ties to the lower centroid id). A CTA
// holds 64 rows and walks all centroids in tiles of 64; each thread keeps the
// running best of its 4 rows over its 4 centroid columns, and the 16 threads
// that share a row reduce at the end with shuffles.
__global__ void __launch_bounds__(256) nearest_centroid_kernel(const float *__restrict__ x, int64_t n, int32_t d,
                                                               const float *__restrict__ c, int32_t nlist,
                                                               int32_t *__restrict__ assign, float *__restrict__ best) {
    __shared__ __align__(16) float Xs[32][68];
    __shared__ __align__(16) float Cs[32][68];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int64_t r0 = (int64_t)blockIdx.x * 64;
    float bd[4];
    int bi[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        bd[u] = __int_as_float(0x7f800000);
        bi[u] = 0;  // stays a valid bucket id even if every distance is inf/NaN
    }
    for (int c0 = 0; c0 < nlist; c0 += 64) {
        float acc[4][4] = {};
        for (int j0 = 0; j0 < d; j0 += 32) {
            for (int e = tid; e < 64 * 32; e += 256) {
                int rr = e >> 5, jj = e & 31;
                int64_t r = r0 + rr;
                int j = j0 + jj;
                Xs[jj][rr] = (r < n && j < d) ? x[r * d + j] : 0.f;
                int ci = c0 + rr;
                Cs[jj][rr] = (ci < nlist && j < d) ? c[(int64_t)ci * d + j] : 0.f;
            }
            __syncthreads();
            const int jn = min(32, d - j0);
            for (int jj = 0; jj < jn; ++jj) {
                float4 a = *reinterpret_cast<const float4 *>(&Xs[jj][ty * 4]);
                float4 b = *reinterpret_cast<const float4 *>(&Cs[jj][tx * 4]);
                float aa[4] = {a.x, a.y, a.z, a.w}, bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        float t = aa[u] - bb[v];
                        acc[u][v] = fmaf(t, t, acc[u][v]);
                    }
            }
            __syncthreads();
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                int ci = c0 + tx * 4 + v;
                if (ci < nlist && (acc[u][v] < bd[u] || (acc[u][v] == bd[u] && ci < bi[u]))) {
                    bd[u] = acc[u][v];
                    bi[u] = ci;
                }
            }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int o = 8; o; o >>= 1) {
            float od = __shfl_xor_sync(0xffffffffu, bd[u], o);
            int oi = __shfl_xor_sync(0xffffffffu, bi[u], o);
            if (od < bd[u] || (od == bd[u] && oi < bi[u])) {
                bd[u] = od;
                bi[u] = oi;
            }
        }
        int64_t r = r0 + ty * 4 + u;
        if (tx == 0 && r < n) {
            assign[r] = bi[u];
            if (best) best[r] = bd[u];
        }
    }
}

cudaError_t launch_nearest_centroids(const float *x, int64_t n, int32_t d, const float *centroids, const float *cnorm,
                                     int32_t nlist, int32_t *assign, float *best, cudaStream_t st) {
    (void)cnorm;
    if (n == 0) return cudaSuccess;
    nearest_centroid_kernel<<<(unsigned)((n + 63) / 64), 256, 0, st>>>(x, n, d, centroids, nlist, assign, best);
    return counted(cudaGetLastError());
}

// Lloyd update: per-bucket sums and counts (one warp per row), then means.
__global__ void kmeans_accum_kernel(const float *__restrict__ x, int64_t n, int32_t d, const int32_t *__restrict__ assign,
                                    float *__restrict__ sums, int32_t *__restrict__ counts) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const int a = assign[r];
    for (int j = lane; j < d; j += 32) atomicAdd(sums + (int64_t)a * d + j, x[r * d + j]);
    if (lane == 0) atomicAdd(counts + a, 1);
}

__global__ void kmeans_finalize_kernel(const float *__restrict__ sums, const int32_t *__restrict__ counts, int32_t nlist,
                                       int32_t d, float *__restrict__ c) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nlist * d) return;
    const int cc = (int)(i / d);
    if (counts[cc] > 0) c[i] = sums[i] / (float)counts[cc];  // an empty bucket keeps its centroid
}

cudaError_t launch_kmeans_update(const float *x, int64_t n, int32_t d, const int32_t *assign, int32_t nlist,
                                 float *sums, int32_t *counts, float *centroids, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(sums, 0, (size_t)nlist * d * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, (size_t)nlist * 4, st);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        kmeans_accum_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(x, n, d, assign, sums, counts);
        e = counted(cudaGetLastError());
        if (e != cudaSuccess) return e;
    }
    int64_t tot = (int64_t)nlist * d;
    kmeans_finalize_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(sums, counts, nlist, d, centroids);
    return counted(cudaGetLastError());
}

// probes[q][r] = bucket id of the r-th nearest centroid
__global__ void keys_to_parts_kernel(const uint64_t *topk, int64_t total, int32_t *probes) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    uint64_t key = topk[i];
    probes[i] = (key == kEmptyKey) ? -1 : key_id(key);
}

cudaError_t launch_keys_to_parts(const uint64_t *topk, int64_t nq, int32_t nprobe, int32_t *probes, cudaStream_t st) {
    int64_t total = nq * nprobe;
    if (total == 0) return cudaSuccess;
    keys_to_parts_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(topk, total, probes);
    return counted(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// BSA metadata. chk[t] = dimensions visited at the t-th prune check.
// resid[b][t][lane] = sum_{j >= chk[t]} x[b][j][lane]^2 (unvisited energy of
// each stored vector); qaux[q][t] = (sum_{j >= chk[t]} q_j^2, F(chk[t])) with
// F(d) = sum_{j < d} var_j / sum_j var_j (1 without variances: the
// Cauchy-Schwarz inner-product bound uses the norms alone).
__global__ void bsa_resid_kernel(const float *__restrict__ data, int64_t nblocks, int32_t d,
                                 const int32_t *__restrict__ chk, int32_t nchk, float *__restrict__ resid) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nblocks * kBlock) return;
    const int64_t b = t / kBlock;
    const int lane = (int)(t % kBlock);
    const float *xb = data + b * d * kBlock + lane;
    float s = 0.f;
    int c = nchk - 1;
    for (int j = d - 1; j >= 0 && c >= 0; --j) {
        float v = xb[(int64_t)j * kBlock];
        s = fmaf(v, v, s);
        while (c >= 0 && chk[c] == j) {
            resid[(b * nchk + c) * kBlock + lane] = s;
            --c;
        }
    }
}

cudaError_t launch_bsa_resid(const float *data, const int32_t *blk_cnt, int64_t nblocks, int32_t d, const int32_t *chk,
                             int32_t nchk, float *resid, cudaStream_t st) {
    (void)blk_cnt;
    if (nblocks == 0 || nchk == 0) return cudaSuccess;
    int64_t th = nblocks * kBlock;
    bsa_resid_kernel<<<(unsigned)((th + 255) / 256), 256, 0, st>>>(data, nblocks, d, chk, nchk, resid);
    return counted(cudaGetLastError());
}

__global__ void bsa_qaux_kernel(const float *__restrict__ q, int64_t nq, int32_t d, const float *__restrict__ var,
                                const int32_t *__restrict__ chk, int32_t nchk, float *__restrict__ qaux) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nq) return;
    const float *qr = q + r * d;
    float tot = 0.f;
    if (var)
        for (int j = 0; j < d; ++j) tot += var[j];
    float s1 = 0.f, sv = 0.f;
    int c = nchk - 1;
    for (int j = d - 1; j >= 0 && c >= 0; --j) {
        float v = qr[j];
        s1 = fmaf(v, v, s1);
        if (var) sv += var[j];
        while (c >= 0 && chk[c] == j) {
            qaux[(r * nchk + c) * 2] = s1;                                   // ||q_r||^2
            qaux[(r * nchk + c) * 2 + 1] = tot > 0.f ? 1.f - sv / tot : 1.f;  // F(d): visited variance fraction
            --c;
        }
    }
}

cudaError_t launch_bsa_qaux(const float *q, int64_t nq, int32_t d, const float *var, const int32_t *chk, int32_t nchk,
                            float *qaux, cudaStream_t st) {
    if (nq == 0 || nchk == 0) return cudaSuccess;
    bsa_qaux_kernel<<<(unsigned)((nq + 127) / 128), 128, 0, st>>>(q, nq, d, var, chk, nchk, qaux);
    return counted(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// PCA for BSA. Column sums and the cross-product matrix X^T X of a sample, in
// FP64 (64x64 output tiles over 32-row chunks).
__global__ void __launch_bounds__(256) gram_kernel(const float *__restrict__ x, int64_t n, int32_t d,
                                                   double *__restrict__ gram) {
    __shared__ double As[32][64];
    __shared__ double Bs[32][64];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
    double acc[4][4] = {};
    for (int64_t r0 = (int64_t)blockIdx.z * 32; r0 < n; r0 += (int64_t)gridDim.z * 32) {
        for (int e = tid; e < 32 * 64; e += 256) {
            int rr = e >> 6, cc = e & 63;
            int64_t r = r0 + rr;
            As[rr][cc] = (r < n && i0 + cc < d) ? (double)x[r * d + i0 + cc] : 0.0;
            Bs[rr][cc] = (r < n && j0 + cc < d) ? (double)x[r * d + j0 + cc] : 0.0;
        }
        __syncthreads();
        for (int rr = 0; rr < 32; ++rr) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += As[rr][ty * 4 + u] * Bs[rr][tx * 4 + v];
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int i = i0 + ty * 4 + u, j = j0 + tx * 4 + v;
            if (i < d && j < d) atomicAdd(gram + (int64_t)i * d + j, acc[u][v]);
        }
}

__global__ void colsum_kernel(const float *__restrict__ x, int64_t n, int32_t d, double *__restrict__ sum) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    double s = 0.0;
    for (int64_t r = blockIdx.y; r < n; r += gridDim.y) s += (double)x[r * d + j];
    atomicAdd(sum + j, s);
}

cudaError_t launch_column_stats(const float *x, int64_t n, int32_t d, double *sum, double *gram, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(sum, 0, (size_t)d * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(gram, 0, (size_t)d * d * 8, st);
    if (e != cudaSuccess) return e;
    dim3 g1((unsigned)((d + 127) / 128), 64);
    colsum_kernel<<<g1, 128, 0, st>>>(x, n, d, sum);
    e = counted(cudaGetLastError());
    if (e != cudaSuccess) return e;
    dim3 g2((unsigned)((d + 63) / 64), (unsigned)((d + 63) / 64), 16);
    gram_kernel<<<g2, 256, 0, st>>>(x, n, d, gram);
    return counted(cudaGetLastError());
}

// Parallel cyclic Jacobi eigen-decomposition of a symmetric FP64 matrix
// (Brent-Luk round-robin ordering: d/2 disjoint (p, q) pairs per step, d-1
// steps per sweep). One step: each pair's rotation (c, s) zeroes A[p][q];
// A <- J^T A J and V <- V J are applied element-wise from the old A.
__device__ __forceinline__ int rr_player(int pos, int round, int m) {
    // m players (even); player 0 fixed, the others rotate by `round`
    return pos == 0 ? 0 : 1 + (pos - 1 + round) % (m - 1);
}

__global__ void jacobi_angles_kernel(const double *__restrict__ A, int32_t dd, int32_t m, int round,
                                     int32_t *__restrict__ partner, double *__restrict__ cs) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;  // pair index
    if (k >= m / 2) return;
    int p = rr_player(k, round, m), q = rr_player(m - 1 - k, round, m);
    if (p > q) {
        int t = p;
        p = q;
        q = t;
    }
    double c = 1.0, s = 0.0;
    if (q < dd) {
        double apq = A[(int64_t)p * dd + q];
        if (apq != 0.0) {
            double app = A[(int64_t)p * dd + p], aqq = A[(int64_t)q * dd + q];
            double theta = (aqq - app) / (2.0 * apq);
            double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
        }
    }
    // index i pairs with partner[i]; cs[i] = (c, s) and a role sign: for p the
    // rotated column is c*a_p - s*a_q, for q it is s*a_p + c*a_q
    if (p < dd) {
        partner[p] = q < dd ? q : -1;
        cs[2 * p] = c;
        cs[2 * p + 1] = -s;
    }
    if (q < dd) {
        partner[q] = p;
        cs[2 * q] = c;
        cs[2 * q + 1] = s;
    }
}

// new[i][j] = sum over a in {i, i'} and b in {j, j'} of J[a][i] A[a][b] J[b][j]
// with J[i][i] = c_i, J[i'][i] = coefficient of the partner in column i.
__global__ void jacobi_apply_kernel(const double *__restrict__ A, double *__restrict__ An, const double *__restrict__ V,
                                    double *__restrict__ Vn, int32_t dd, const int32_t *__restrict__ partner,
                                    const double *__restrict__ cs) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)dd * dd) return;
    const int i = (int)(t / dd), j = (int)(t % dd);
    const int pi = partner[i], pj = partner[j];
    const double ci = cs[2 * i], si = cs[2 * i + 1], cj = cs[2 * j], sj = cs[2 * j + 1];
    // column i of AJ: c_i * A[:, i] + s_i * A[:, pi]
    double v = ci * cj * A[(int64_t)i * dd + j];
    if (pj >= 0) v += ci * sj * A[(int64_t)i * dd + pj];
    if (pi >= 0) {
        v += si * cj * A[(int64_t)pi * dd + j];
        if (pj >= 0) v += si * sj * A[(int64_t)pi * dd + pj];
    }
    An[t] = v;
    double w = cj * V[(int64_t)i * dd + j];
    if (pj >= 0) w += sj * V[(int64_t)i * dd + pj];
    Vn[t] = w;
}

__global__ void offdiag_kernel(const double *__restrict__ A, int32_t dd, double *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (t < (int64_t)dd * dd) {
        int i = (int)(t / dd), j = (int)(t % dd);
        double a = A[t];
        v = (i != j) ? a * a : 0.0;
    }
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(out, v);
}

// Eigen-decomposition of the symmetric dd x dd matrix in A (device, FP64,
// overwritten). On return A's diagonal holds the eigenvalues and V (device,
// FP64) the eigenvectors as columns. work: 2*dd*dd + 3*(dd+1) doubles.
cudaError_t jacobi_eigen(double *A, double *V, int32_t dd, double *work, int sweeps, cudaStream_t st) {
    const int m = dd + (dd & 1);
    double *bufA = work, *bufV = work + (size_t)dd * dd;
    double *cs = bufV + (size_t)dd * dd;
    int32_t *partner = reinterpret_cast<int32_t *>(cs + 2 * (size_t)(dd + 1));
    const int64_t tot = (int64_t)dd * dd;
    const unsigned g = (unsigned)((tot + 255) / 256);
    double *curA = A, *curV = V, *nxtA = bufA, *nxtV = bufV;
    for (int sweep = 0; sweep < sweeps; ++sweep) {
        for (int round = 0; round < m - 1; ++round) {
            jacobi_angles_kernel<<<(m / 2 + 127) / 128, 128, 0, st>>>(curA, dd, m, round, partner, cs);
            cudaError_t e = counted(cudaGetLastError());
            if (e != cudaSuccess) return e;
            jacobi_apply_kernel<<<g, 256, 0, st>>>(curA, nxtA, curV, nxtV, dd, partner, cs);
            e = counted(cudaGetLastError());
            if (e != cudaSuccess) return e;
            double *t = curA; curA = nxtA; nxtA = t;
            t = curV; curV = nxtV; nxtV = t;
        }
    }
    if (curA != A) {
        cudaError_t e = cudaMemcpyAsync(A, curA, (size_t)tot * 8, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(V, curV, (size_t)tot * 8, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_offdiag(const double *A, int32_t dd, double *out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, 8, st);
    if (e != cudaSuccess) return e;
    int64_t tot = (int64_t)dd * dd;
    offdiag_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(A, dd, out);
    return counted(cudaGetLastError());
}

}  // namespace pdx
