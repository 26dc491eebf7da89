// SH codebook (Sec. 3.3: the SH coefficients, about 3/4 of a model's size,
// are clustered with K-means across all layers; Sec. 4.3).  Lloyd's
// iteration on the device, then encoding: every Gaussian keeps its DC
// coefficient and stores a 16-bit index into an FP16 table of the remaining
// 3(K-1) coefficients.  The preprocess gathers those rows from L2 instead of
// reading 3(K-1) floats per Gaussian from HBM.
//
// Assignment is brute force: a thread per point holds its (zero-padded)
// coordinates in registers and scans the centroids staged in shared memory
// 64 at a time with 16-byte broadcast loads.  Ties go to the lower index.
#include <cuda_fp16.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kKmTile = 64;                  // centroids per shared-memory tile
constexpr int kKmThreads = 128;

__global__ void __launch_bounds__(kKmThreads) k_kmeans_assign(const float *__restrict__ pts, int64_t n, int dim,
                                                              int64_t stride, const float *__restrict__ cent, int k,
                                                              uint32_t *__restrict__ assign) {
    __shared__ float4 s_c[kKmTile][kCbMaxDim / 4];
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kKmThreads + threadIdx.x;
    float x[kCbMaxDim];
#pragma unroll
    for (int d = 0; d < kCbMaxDim; ++d) x[d] = (i < n && d < dim) ? pts[i * stride + d] : 0.f;
    float best = 3.0e38f;
    uint32_t arg = 0;
    for (int t0 = 0; t0 < k; t0 += kKmTile) {
        __syncthreads();
        for (int e = threadIdx.x; e < kKmTile * kCbMaxDim; e += kKmThreads) {
            const int j = e / kCbMaxDim, d = e % kCbMaxDim;
            reinterpret_cast<float *>(&s_c[j][0])[d] = (t0 + j < k && d < dim) ? cent[(t0 + j) * dim + d] : 0.f;
        }
        __syncthreads();
        const int m = min(kKmTile, k - t0);
        for (int j = 0; j < m; ++j) {
            float acc = 0.f;
#pragma unroll
            for (int q = 0; q < kCbMaxDim / 4; ++q) {
                const float4 c = s_c[j][q];
                const float a = x[4 * q] - c.x, b = x[4 * q + 1] - c.y, e = x[4 * q + 2] - c.z, f = x[4 * q + 3] - c.w;
                acc = fmaf(a, a, acc);
                acc = fmaf(b, b, acc);
                acc = fmaf(e, e, acc);
                acc = fmaf(f, f, acc);
            }
            if (acc < best) {
                best = acc;
                arg = static_cast<uint32_t>(t0 + j);
            }
        }
    }
    if (i < n) assign[i] = arg;
}

__global__ void __launch_bounds__(256) k_kmeans_accumulate(const float *__restrict__ pts, int64_t n, int dim,
                                                           int64_t stride, const uint32_t *__restrict__ assign,
                                                           float *__restrict__ sums, float *__restrict__ cnt) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint32_t a = assign[i];
        for (int d = 0; d < dim; ++d) atomicAdd(&sums[static_cast<size_t>(a) * dim + d], pts[i * stride + d]);
        atomicAdd(&cnt[a], 1.f);
    }
}

__global__ void __launch_bounds__(256) k_kmeans_finish(const float *__restrict__ sums, const float *__restrict__ cnt,
                                                       int k, int dim, float *__restrict__ cent) {
    const int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (e >= static_cast<int64_t>(k) * dim) return;
    const float c = cnt[e / dim];
    if (c > 0.f) cent[e] = sums[e] / c;
}

// DC copy, 16-bit indices and the FP16 table (rows padded to `row` halves).
__global__ void __launch_bounds__(256) k_sh_encode(const float *__restrict__ sh, int64_t n, int K,
                                                   const uint32_t *__restrict__ assign, const float *__restrict__ cent,
                                                   int k, int row, float *__restrict__ dc,
                                                   uint16_t *__restrict__ index, __half *__restrict__ table) {
    const int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    const int dim = 3 * (K - 1);
    if (e < n) {
        dc[3 * e] = sh[e * 3 * K];
        dc[3 * e + 1] = sh[e * 3 * K + 1];
        dc[3 * e + 2] = sh[e * 3 * K + 2];
        index[e] = static_cast<uint16_t>(assign[e]);
    }
    if (e < static_cast<int64_t>(k) * row) {
        const int64_t j = e / row, d = e % row;
        table[e] = __float2half_rn(d < dim ? cent[j * dim + d] : 0.f);
    }
}

}  // namespace

cudaError_t launch_kmeans_assign(const float *pts, int64_t n, int dim, int64_t stride, const float *cent, int k,
                                 uint32_t *assign, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_kmeans_assign<<<static_cast<unsigned>((n + kKmThreads - 1) / kKmThreads), kKmThreads, 0, st>>>(pts, n, dim, stride,
                                                                                                  cent, k, assign);
    return cudaGetLastError();
}

cudaError_t launch_kmeans_update(const float *pts, int64_t n, int dim, int64_t stride, const uint32_t *assign, int k,
                                 float *cent, float *scratch, cudaStream_t st) {
    float *sums = scratch, *cnt = scratch + static_cast<size_t>(k) * dim;
    cudaError_t e = cudaMemsetAsync(scratch, 0, static_cast<size_t>(k) * (dim + 1) * sizeof(float), st);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        const int blocks = static_cast<int>(std::min<int64_t>((n + 255) / 256, 8 * 1024));
        k_kmeans_accumulate<<<blocks, 256, 0, st>>>(pts, n, dim, stride, assign, sums, cnt);
    }
    const int64_t tot = static_cast<int64_t>(k) * dim;
    k_kmeans_finish<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, st>>>(sums, cnt, k, dim, cent);
    return cudaGetLastError();
}

cudaError_t launch_sh_encode(const float *sh, int64_t n, int K, const uint32_t *assign, const float *cent, int k,
                             float *dc, uint16_t *index, void *table, cudaStream_t st) {
    const int row = cb_row_halves(K);
    const int64_t tot = std::max<int64_t>(n, static_cast<int64_t>(k) * row);
    if (tot == 0) return cudaSuccess;
    k_sh_encode<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, st>>>(sh, n, K, assign, cent, k, row, dc, index,
                                                                       static_cast<__half *>(table));
    return cudaGetLastError();
}

}  // namespace gs
